"""Seeded synthetic crystals that stand in for the paper's DFT force constants.

This module is the input recipe shared by the tests, the benchmark and the oracle
harness.  It builds, from a seed, a lattice, a basis, masses, harmonic pair force
constants (Phi2, eV/A^2) and fourth-order force constants (Phi4, eV/A^4) in the
quartet-list form consumed by the library (atom i in the home cell; atoms j, k, l
with integer cell vectors).  It holds none of the scattering-rate arithmetic.

Recipe (the paper's materials are Si, BAs and LiCoO2, Sec. 3; their DFT force
constants are replaced by spring models of the same structures and masses):

* Phi2: per bond (atom i in cell 0, atom j in cell R, separation d) a spring block
  -(k_c dd^T/|d|^2 + k_t (I - dd^T/|d|^2)); the self block is minus the sum of
  the pair blocks, so the acoustic sum rule holds exactly.
* Phi4: per unordered nearest-neighbour bond a 3^4 tensor K with entries drawn
  N(0, 5 eV/A^4), averaged over the 24 index permutations (the transposition
  symmetry of Sec. 2.3, Eq. TS).  It enters as the fourth derivative of the bond
  energy K (u_b - u_a)^4 / 4!, i.e. the quartet over sites (x1..x4) in {a, b}^4
  gets s1 s2 s3 s4 K with s = -1 on site a and +1 on site b.  Summing over any
  site index gives zero (the acoustic sum rule of Sec. 2.3, Eq. ASR).
* Phi4, general form (`general=True`, parity tests only): per bond a 6^4 tensor over the
  six displacement components of its two sites, entries N(0, 5 eV/A^4), averaged over
  the 24 permutations of its four axes.  The quartet over sites (x1..x4) gets the
  block of the tensor at those sites.  This keeps the transposition symmetry of
  Eq. TS but, unlike the bond energy above, is not symmetric in the Cartesian indices
  of one quartet alone (so a transposed Cartesian index changes the vertex), and it
  does not obey the acoustic sum rule.
* Seeds: numpy PCG64 with seed 2104_04895 + config index.

The five workloads follow the published benchmark table of the method's build
(simple cubic, diamond Si-like, zincblende BAs-like, rhombohedral LiCoO2-like,
dense Si-like temperature sweep).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2104_04895


@dataclass
class Crystal:
    name: str
    lattice: np.ndarray          # (3,3) rows a1, a2, a3 in Angstrom
    frac: np.ndarray             # (natoms,3) fractional positions
    mass: np.ndarray             # (natoms,) amu
    fc2_idx: np.ndarray          # (n2,5) int32: i, j, R[3]
    fc2_val: np.ndarray          # (n2,9) float64, eV/A^2, row-major alpha,beta
    fc4_idx: np.ndarray          # (n4,13) int32: i, j, k, l, Rj[3], Rk[3], Rl[3]
    fc4_val: np.ndarray          # (n4,81) float64, eV/A^4, row-major alpha..theta
    grid: tuple = (4, 4, 4)
    temps: tuple = (300.0,)
    scalebroad: float = 1.0
    extra: dict = field(default_factory=dict)
    fc3_idx: np.ndarray = None   # (n3,9) int32: i, j, k, Rj[3], Rk[3]
    fc3_val: np.ndarray = None   # (n3,27) float64, eV/A^3, row-major alpha,beta,gamma

    @property
    def natoms(self) -> int:
        return int(self.mass.shape[0])

    @property
    def nb(self) -> int:
        return 3 * self.natoms

    @property
    def nq(self) -> int:
        return int(np.prod(self.grid))

    def with_grid(self, grid, temps=None) -> "Crystal":
        c = Crystal(self.name, self.lattice, self.frac, self.mass, self.fc2_idx, self.fc2_val,
                    self.fc4_idx, self.fc4_val, tuple(int(g) for g in grid),
                    tuple(temps) if temps is not None else self.temps, self.scalebroad, dict(self.extra),
                    self.fc3_idx, self.fc3_val)
        return c

    def scaled_fc4(self, s: float) -> "Crystal":
        c = self.with_grid(self.grid)
        c.fc4_val = self.fc4_val * s
        return c


# --------------------------------------------------------------------------- geometry
def _cart(lattice, frac):
    return np.asarray(frac, dtype=np.float64) @ lattice


def _neighbours(lattice, frac, rmax, span=3):
    """All (i, j, R, d) with i in cell 0, |d| <= rmax, d = x_j + R - x_i (Cartesian)."""
    out = []
    nat = len(frac)
    xs = _cart(lattice, frac)
    rng = range(-span, span + 1)
    for i in range(nat):
        for j in range(nat):
            for R in itertools.product(rng, rng, rng):
                if i == j and R == (0, 0, 0):
                    continue
                d = xs[j] + np.asarray(R, float) @ lattice - xs[i]
                r = float(np.linalg.norm(d))
                if r <= rmax + 1e-9:
                    out.append((i, j, tuple(int(v) for v in R), d, r))
    return out


def _fc2_springs(lattice, frac, shells):
    """shells: list of (rmin, rmax, kc_fn, kt_fn) where k*_fn(i, j, d) -> spring constant."""
    nat = len(frac)
    rmax = max(s[1] for s in shells)
    blocks = {}
    for (i, j, R, d, r) in _neighbours(lattice, frac, rmax):
        for (lo, hi, kc_fn, kt_fn) in shells:
            if lo - 1e-6 <= r <= hi + 1e-6:
                u = d / r
                P = np.outer(u, u)
                kc, kt = kc_fn(i, j, d), kt_fn(i, j, d)
                blk = -(kc * P + kt * (np.eye(3) - P))
                key = (i, j, R)
                blocks[key] = blocks.get(key, np.zeros((3, 3))) + blk
                self_key = (i, i, (0, 0, 0))
                blocks[self_key] = blocks.get(self_key, np.zeros((3, 3))) - blk
                break
    keys = sorted(blocks)
    idx = np.array([[k[0], k[1], *k[2]] for k in keys], dtype=np.int32)
    val = np.array([blocks[k].reshape(9) for k in keys], dtype=np.float64)
    return idx, val


def _sym24(K):
    """Average a 3^4 tensor over the 24 permutations of its indices."""
    acc = np.zeros_like(K)
    for p in itertools.permutations(range(4)):
        acc += np.transpose(K, p)
    return acc / 24.0


def _bonds_unordered(lattice, frac, pair_ok, rmax):
    """Unordered bonds, one per translation class: (a, b, R, d) with a <= b."""
    out = []
    for (i, j, R, d, r) in _neighbours(lattice, frac, rmax):
        if not pair_ok(i, j, d, r):
            continue
        if i < j or (i == j and R > (0, 0, 0)):
            out.append((i, j, R, d))
    return out


def _fc4_from_bonds(bonds, tensors):
    """Quartet list from bond tensors: sites {a@0, b@R}^4, shifted so the first atom is in cell 0."""
    acc = {}
    for (a, b, R, _d), K in zip(bonds, tensors):
        sites = [(a, (0, 0, 0), -1.0), (b, tuple(R), +1.0)]
        for combo in itertools.product(sites, repeat=4):
            sgn = combo[0][2] * combo[1][2] * combo[2][2] * combo[3][2]
            c0 = np.asarray(combo[0][1])
            atoms = tuple(s[0] for s in combo)
            cells = tuple(tuple(int(v) for v in (np.asarray(s[1]) - c0)) for s in combo[1:])
            key = (atoms, cells)
            acc[key] = acc.get(key, np.zeros((3, 3, 3, 3))) + sgn * K
    keys = sorted(acc)
    idx = np.array([[*k[0], *k[1][0], *k[1][1], *k[1][2]] for k in keys], dtype=np.int32)
    val = np.array([acc[k].reshape(81) for k in keys], dtype=np.float64)
    return idx, val


def _draw_pair_tensors(rng, n, scale=5.0):
    """Per bond a 6^4 tensor over the (site, Cartesian) components of its two sites, N(0, scale) entrywise,
    averaged over the 24 permutations of its axes."""
    out = []
    for _ in range(n):
        T = rng.normal(0.0, scale, size=(6, 6, 6, 6))
        out.append(sum(np.transpose(T, p) for p in itertools.permutations(range(4))) / 24.0)
    return out


def _fc4_from_pair_tensors(bonds, tensors):
    """Quartet list from per-bond 6^4 tensors: the quartet over sites (x1..x4) in {a@0, b@R}^4 gets the 3^4 block
    of the tensor at those sites, shifted so the first atom is in cell 0."""
    acc = {}
    for (a, b, R, _d), T in zip(bonds, tensors):
        T8 = T.reshape(2, 3, 2, 3, 2, 3, 2, 3)
        sites = [(a, (0, 0, 0), 0), (b, tuple(R), 1)]
        for combo in itertools.product(sites, repeat=4):
            c0 = np.asarray(combo[0][1])
            atoms = tuple(s[0] for s in combo)
            cells = tuple(tuple(int(v) for v in (np.asarray(s[1]) - c0)) for s in combo[1:])
            key = (atoms, cells)
            blk = T8[combo[0][2], :, combo[1][2], :, combo[2][2], :, combo[3][2], :]
            acc[key] = acc.get(key, np.zeros((3, 3, 3, 3))) + blk
    keys = sorted(acc)
    idx = np.array([[*k[0], *k[1][0], *k[1][1], *k[1][2]] for k in keys], dtype=np.int32)
    val = np.array([acc[k].reshape(81) for k in keys], dtype=np.float64)
    return idx, val


def _fc4(bonds, rng, general):
    """Phi4 quartets of the bonds: the bond-energy form, or the general per-bond form (see the module notes)."""
    if general:
        return _fc4_from_pair_tensors(bonds, _draw_pair_tensors(rng, len(bonds)))
    return _fc4_from_bonds(bonds, _draw_tensors(rng, len(bonds)))


def _fc3_from_bonds(bonds, tensors):
    """Triplet list from third-order bond tensors: sites {a@0, b@R}^3 with the sign product of the bond's ends
    (-1 at a, +1 at b: the derivatives of K (u_b - u_a)^3 / 6), shifted so the first atom is in cell 0. Each
    index sums to zero over the other two (acoustic sum rule) by construction."""
    acc = {}
    for (a, b, R, _d), K in zip(bonds, tensors):
        sites = [(a, (0, 0, 0), -1.0), (b, tuple(R), +1.0)]
        for combo in itertools.product(sites, repeat=3):
            sgn = combo[0][2] * combo[1][2] * combo[2][2]
            c0 = np.asarray(combo[0][1])
            atoms = tuple(s[0] for s in combo)
            cells = tuple(tuple(int(v) for v in (np.asarray(s[1]) - c0)) for s in combo[1:])
            key = (atoms, cells)
            acc[key] = acc.get(key, np.zeros((3, 3, 3))) + sgn * K
    keys = sorted(acc)
    idx = np.array([[*k[0], *k[1][0], *k[1][1]] for k in keys], dtype=np.int32)
    val = np.array([acc[k].reshape(27) for k in keys], dtype=np.float64)
    return idx, val


def _draw_fc3(bonds, seed_index, scale=5.0):
    """Seeded third-order bond tensors, N(0, scale eV/A^3) entrywise, averaged over index permutations; drawn
    from their own stream so that the fourth-order draws do not change."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1000 + seed_index))
    out = []
    for _ in bonds:
        K = rng.normal(0.0, scale, size=(3, 3, 3))
        out.append(sum(np.transpose(K, p) for p in itertools.permutations(range(3))) / 6.0)
    return _fc3_from_bonds(bonds, out)


def _draw_tensors(rng, n, scale=5.0):
    return [_sym24(rng.normal(0.0, scale, size=(3, 3, 3, 3))) for _ in range(n)]


def _rot4(g, K):
    return np.einsum("ai,bj,ck,dl,ijkl->abcd", g, g, g, g, K)


def _signed_perms():
    ops = []
    for p in itertools.permutations(range(3)):
        for s in itertools.product((1, -1), repeat=3):
            g = np.zeros((3, 3))
            for r in range(3):
                g[r, p[r]] = s[r]
            ops.append(g)
    return ops


def _point_group_tensors(bond_vecs, tensors, ops):
    """Average each bond tensor over the point group acting on the bond vectors.

    bond_vecs: Cartesian vectors of the unordered bonds (a K for -d equals that for d).
    Returns tensors invariant under every op in `ops` (which must map the bond set to itself).
    """
    def find(v):
        for n, d in enumerate(bond_vecs):
            if np.allclose(v, d, atol=1e-8) or np.allclose(v, -d, atol=1e-8):
                return n
        raise ValueError("op does not map the bond set to itself")
    out = []
    for d in bond_vecs:
        acc = np.zeros((3, 3, 3, 3))
        for g in ops:
            src = find(g.T @ d)          # g^{-1} d
            acc += _rot4(g, tensors[src])
        out.append(acc / len(ops))
    return out


# --------------------------------------------------------------------------- structures
def simple_cubic(grid=(4, 4, 4), seed_index=1, symmetric=False, temps=(300.0,), scalebroad=1.0, general=False):
    """Simple cubic monatomic, a = 3.0 A, 28.0855 amu, central NN k1=1.0, NNN k2=0.5 eV/A^2.  general=True draws
    the general per-bond Phi4 (module notes) instead of the bond-energy form."""
    a = 3.0
    lattice = np.eye(3) * a
    frac = np.zeros((1, 3))
    mass = np.array([28.0855])
    shells = [(a, a, lambda i, j, d: 1.0, lambda i, j, d: 0.0),
              (a * np.sqrt(2), a * np.sqrt(2), lambda i, j, d: 0.5, lambda i, j, d: 0.0)]
    i2, v2 = _fc2_springs(lattice, frac, shells)
    bonds = _bonds_unordered(lattice, frac, lambda i, j, d, r: abs(r - a) < 1e-6, a)
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_index))
    extra = {}
    if general:
        if symmetric:
            raise ValueError("the general Phi4 form is not point-group averaged")
        i4, v4 = _fc4(bonds, rng, True)
    else:
        K = _draw_tensors(rng, len(bonds))
        if symmetric:
            K = _point_group_tensors([b[3] for b in bonds], K, _signed_perms())
            extra["point_group"] = _signed_perms()
        i4, v4 = _fc4_from_bonds(bonds, K)
    i3, v3 = _draw_fc3(bonds, seed_index)
    name = "simple-cubic" + ("-sym" if symmetric else "") + ("-gen" if general else "")
    return Crystal(name, lattice, frac, mass, i2, v2, i4, v4, tuple(grid), tuple(temps), scalebroad, extra, i3, v3)


def _fcc_two_atom(a, masses, name, grid, seed_index, symmetric, temps, scalebroad, general=False):
    lattice = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    frac = np.array([[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]])
    mass = np.asarray(masses, dtype=np.float64)
    r1 = a * np.sqrt(3.0) / 4.0
    r2 = a / np.sqrt(2.0)
    shells = [(r1, r1, lambda i, j, d: 1.0, lambda i, j, d: 0.25),
              (r2, r2, lambda i, j, d: 0.5, lambda i, j, d: 0.125)]
    i2, v2 = _fc2_springs(lattice, frac, shells)
    bonds = _bonds_unordered(lattice, frac, lambda i, j, d, r: abs(r - r1) < 1e-6, r1)
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_index))
    extra = {}
    if general:
        if symmetric:
            raise ValueError("the general Phi4 form is not point-group averaged")
        i4, v4 = _fc4(bonds, rng, True)
    else:
        K = _draw_tensors(rng, len(bonds))
        if symmetric:
            vecs = [b[3] for b in bonds]
            ops = [g for g in _signed_perms()
                   if all(any(np.allclose(g @ d, e, atol=1e-8) for e in vecs) for d in vecs)]
            K = _point_group_tensors(vecs, K, ops)
            extra["point_group"] = ops
        i4, v4 = _fc4_from_bonds(bonds, K)
    i3, v3 = _draw_fc3(bonds, seed_index)
    return Crystal(name + ("-sym" if symmetric else "") + ("-gen" if general else ""), lattice, frac, mass, i2, v2,
                   i4, v4, tuple(grid), tuple(temps), scalebroad, extra, i3, v3)


def diamond_si(grid=(8, 8, 8), seed_index=2, symmetric=False, temps=(300.0,), scalebroad=1.0, general=False):
    """Diamond Si-like: a = 5.43 A, 2 x 28.0855 amu, NN+NNN central and transverse springs."""
    return _fcc_two_atom(5.43, [28.0855, 28.0855], "diamond-si", grid, seed_index, symmetric,
                         temps, scalebroad, general)


def zincblende_bas(grid=(12, 12, 12), seed_index=3, temps=(300.0,), scalebroad=1.0, general=False):
    """Zincblende BAs-like: a = 4.78 A, B 10.81 and As 74.92 amu (large acoustic-optical gap)."""
    return _fcc_two_atom(4.78, [10.81, 74.92], "zincblende-bas", grid, seed_index, False,
                         temps, scalebroad, general)


def licoo2(grid=(10, 10, 6), seed_index=4, temps=(300.0, 500.0, 700.0), scalebroad=1.0, general=False):
    """Rhombohedral layered LiCoO2-like (R-3m), 4 atoms: Li, Co, O, O.

    a_hex = 2.82 A, c_hex = 14.05 A, O at +-(u,u,u) with u = 0.26.  Springs: bonds
    within 1.2x the shortest cation-O distance plus in-plane metal-metal bonds;
    in-plane bonds (|d_z|/|d| < 0.5) k_c = 3.0, interlayer k_c = 1.0 eV/A^2, and a
    transverse part 0.25 k_c.  Phi4 on the cation-O bonds (Co-O and Li-O, the
    nearest-neighbour shell of each cation).
    """
    ah, ch, u = 2.82, 14.05, 0.26
    lattice = np.array([[ah / 2, -ah / (2 * np.sqrt(3)), ch / 3],
                        [0.0, ah / np.sqrt(3), ch / 3],
                        [-ah / 2, -ah / (2 * np.sqrt(3)), ch / 3]])
    frac = np.array([[0.5, 0.5, 0.5], [0.0, 0.0, 0.0], [u, u, u], [-u, -u, -u]])
    mass = np.array([6.94, 58.93, 16.00, 16.00])
    is_cat = [True, True, False, False]
    nb = _neighbours(lattice, frac, 4.0)
    d_co = min(r for (i, j, R, d, r) in nb if is_cat[i] != is_cat[j])
    d_mm = min(r for (i, j, R, d, r) in nb if is_cat[i] and is_cat[j] and i == j)

    def k_of(d):
        return 3.0 if abs(d[2]) / np.linalg.norm(d) < 0.5 else 1.0

    def cat_o(i, j, d, r):
        return is_cat[i] != is_cat[j] and r <= 1.2 * d_co + 1e-9

    def mm(i, j, d, r):
        return is_cat[i] and is_cat[j] and i == j and abs(r - d_mm) < 1e-6

    pairs = {}
    for (i, j, R, d, r) in nb:
        if cat_o(i, j, d, r) or mm(i, j, d, r):
            blk = -(k_of(d) * np.outer(d, d) / r**2 + 0.25 * k_of(d) * (np.eye(3) - np.outer(d, d) / r**2))
            pairs[(i, j, R)] = pairs.get((i, j, R), np.zeros((3, 3))) + blk
            pairs[(i, i, (0, 0, 0))] = pairs.get((i, i, (0, 0, 0)), np.zeros((3, 3))) - blk
    keys = sorted(pairs)
    i2 = np.array([[k[0], k[1], *k[2]] for k in keys], dtype=np.int32)
    v2 = np.array([pairs[k].reshape(9) for k in keys], dtype=np.float64)
    bonds = _bonds_unordered(lattice, frac, cat_o, 1.2 * d_co)
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_index))
    i4, v4 = _fc4(bonds, rng, general)
    i3, v3 = _draw_fc3(bonds, seed_index)
    return Crystal("licoo2" + ("-gen" if general else ""), lattice, frac, mass, i2, v2, i4, v4, tuple(grid),
                   tuple(temps), scalebroad, {}, i3, v3)


TEMPS_SWEEP = tuple(float(t) for t in range(300, 1001, 100))


def point_group_ops(cryst: Crystal) -> np.ndarray:
    """The Cartesian point-group operations a symmetric crystal was built with, as integer matrices acting on
    the reciprocal-lattice fractional coordinates of q (q = f @ B with B the reciprocal vectors as rows):
    R = B^-T g B^T.  Shape (nops, 3, 3), int32."""
    ops = cryst.extra.get("point_group")
    if ops is None:
        raise ValueError(f"{cryst.name} was not built with point-group symmetric force constants")
    B = 2.0 * np.pi * np.linalg.inv(cryst.lattice).T
    out = []
    for g in ops:
        R = np.linalg.inv(B.T) @ g @ B.T
        Ri = np.rint(R)
        if not np.allclose(R, Ri, atol=1e-9):
            raise ValueError("operation is not a lattice symmetry")
        out.append(Ri.astype(np.int32))
    return np.asarray(out, dtype=np.int32)


def workload(index: int) -> Crystal:
    """The five benchmark workloads, 1-based."""
    if index == 1:
        return simple_cubic((4, 4, 4), 1)
    if index == 2:
        return diamond_si((8, 8, 8), 2)
    if index == 3:
        return zincblende_bas((12, 12, 12), 3)
    if index == 4:
        return licoo2((10, 10, 6), 4)
    if index == 5:
        return diamond_si((16, 16, 16), 2, temps=TEMPS_SWEEP)
    raise ValueError(index)


WORKLOAD_NAMES = {
    1: "simple-cubic 4x4x4 nb=3 T=300K sb=1.0",
    2: "diamond-si 8x8x8 nb=6 T=300K sb=1.0",
    3: "zincblende-bas 12x12x12 nb=6 T=300K sb=1.0",
    4: "licoo2 10x10x6 nb=12 T=300/500/700K sb=1.0",
    5: "diamond-si 16x16x16 nb=6 T=300..1000K sb=1.0",
}


# --------------------------------------------------------------------------- random draws shared by tests
def random_modes(nq_grid, nb, seed):
    """Random unit-norm complex vectors and positive frequencies (only for algebraic tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = int(np.prod(nq_grid))
    ev = rng.normal(size=(N, nb, nb)) + 1j * rng.normal(size=(N, nb, nb))
    ev /= np.linalg.norm(ev, axis=2, keepdims=True)
    om = rng.uniform(1.0, 10.0, size=(N, nb))
    return om, ev
