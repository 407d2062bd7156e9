"""Oracle harmonic phonons on the regular q-grid (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this module.  It shares no code with the CUDA path.

Follows the paper's harmonic step (Sec. 2.1: frequencies, eigenvectors and group
velocities from the second-order force constants) with the cell-phase convention
of Eq. V4 (r_j is the position of the unit cell of atom j):

  D_{(i a),(j b)}(q) = sum_R Phi2_{a b}(0 i; R j) exp(i q.R) / sqrt(M_i M_j)
  omega^2 = conv * eig(D)  (conv = eV/(A^2 amu) in ps^-2),  e = unit eigenvectors
  v = d omega / d q = conv * Re(e^H dD/dq e) / (2 omega)   (Hellmann-Feynman)

Readings (where the paper is silent):
  * time reversal is imposed exactly: omega(-q) = omega(q), e(-q) = conj(e(q)),
    v(-q) = -v(q); at a self-conjugate q (q = -q mod G) D is real and e is real,
    so v averages to zero there and is set to zero;
  * the three acoustic modes at Gamma get omega = 0 exactly; any other
    omega^2 < -1e-8 max(omega^2) is an instability;
  * velocities are averaged over degenerate sets (|d omega| <= 1e-8 omega_max),
    i.e. the trace of dD projected on the set, which is gauge invariant.
"""
from __future__ import annotations

import numpy as np

ECHARGE = 1.602176634e-19
AMU = 1.66053906660e-27
CONV = ECHARGE / AMU * 1e20 * 1e-24   # eV/(A^2 amu) -> ps^-2


def grid_points(grid):
    g = np.array([(a, b, c) for a in range(grid[0]) for b in range(grid[1]) for c in range(grid[2])],
                 dtype=np.int64)
    return g


def reciprocal(lattice):
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, float)).T


def dyn_matrix(cryst, gfrac):
    """D(q) and dD/dq (3 Cartesian components) at fractional reciprocal coordinates gfrac."""
    nb = cryst.nb
    D = np.zeros((nb, nb), complex)
    dD = np.zeros((3, nb, nb), complex)
    lat = np.asarray(cryst.lattice, float)
    for idx, val in zip(cryst.fc2_idx, cryst.fc2_val):
        i, j = int(idx[0]), int(idx[1])
        R = idx[2:5].astype(float)
        ph = np.exp(2j * np.pi * float(np.dot(gfrac, R)))
        blk = val.reshape(3, 3) / np.sqrt(cryst.mass[i] * cryst.mass[j])
        D[3 * i:3 * i + 3, 3 * j:3 * j + 3] += blk * ph
        Rc = R @ lat
        for c in range(3):
            dD[c, 3 * i:3 * i + 3, 3 * j:3 * j + 3] += 1j * Rc[c] * blk * ph
    return D, dD


def modes(cryst, degen_tol=1e-8, unstable_tol=1e-8):
    """omega (N,nb) rad/ps, evec (N,nb_branch,nb_comp) complex, vel (N,nb,3) A/ps."""
    grid = cryst.grid
    N, nb = cryst.nq, cryst.nb
    G = grid_points(grid)
    om = np.zeros((N, nb))
    ev = np.zeros((N, nb, nb), complex)
    ve = np.zeros((N, nb, 3))
    done = np.zeros(N, bool)
    ng = np.array(grid)

    def index(g):
        return int((g[0] * grid[1] + g[1]) * grid[2] + g[2])

    for q in range(N):
        if done[q]:
            continue
        g = G[q]
        partner = index((-g) % ng)
        gfrac = g / ng
        D, dD = dyn_matrix(cryst, gfrac)
        selfconj = partner == q
        if selfconj:
            w2, U = np.linalg.eigh(D.real)
            U = U.astype(complex)
        else:
            D = 0.5 * (D + D.conj().T)
            w2, U = np.linalg.eigh(D)
        w2 = w2 * CONV
        wmax2 = max(abs(w2).max(), 1e-300)
        w = np.zeros(nb)
        for b in range(nb):
            if q == 0 and b < 3:
                w[b] = 0.0
            elif w2[b] < -unstable_tol * wmax2:
                raise ValueError(f"unstable mode at q={q} branch={b}: omega^2={w2[b]}")
            else:
                w[b] = np.sqrt(max(w2[b], 0.0))
        # Hellmann-Feynman velocities, averaged over degenerate sets
        raw = np.array([[np.real(U[:, b].conj() @ dD[c] @ U[:, b]) for c in range(3)] for b in range(nb)])
        v = np.zeros((nb, 3))
        wtol = degen_tol * max(w.max(), 1e-300)
        b = 0
        while b < nb:
            e = b + 1
            while e < nb and abs(w[e] - w[e - 1]) <= wtol:
                e += 1
            avg = raw[b:e].mean(axis=0)
            for k in range(b, e):
                v[k] = 0.0 if w[k] == 0.0 else CONV * avg / (2.0 * w[k])
            b = e
        if selfconj:
            v[:] = 0.0
        om[q], ev[q], ve[q] = w, U.T, v
        done[q] = True
        if not selfconj:
            om[partner], ev[partner], ve[partner] = w, U.T.conj(), -v
            done[partner] = True
    return om, ev, ve


def degenerate_sets(omega_row, tol=1e-8):
    wmax = max(omega_row.max(), 1e-300)
    sets, b, nb = [], 0, len(omega_row)
    while b < nb:
        e = b + 1
        while e < nb and abs(omega_row[e] - omega_row[e - 1]) <= tol * wmax:
            e += 1
        sets.append((b, e))
        b = e
    return sets
