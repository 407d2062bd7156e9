"""Pins of the oracle's rates (Eqs. tao0 and 4phgamma, the Gaussian delta of Sec. 2.4).

* a single-q (1x1x1) crystal with injected integer frequencies and zero velocities, where
  only exactly energy-conserving terms enter with delta := 1 (the small-sigma rule of
  Sec. 2.4): the rate is recomputed term by term in SI units from the brute-force
  supercell vertex, which pins the prefactor, the unit conversion, the multiplicities
  1/2, 1/2, 1/6 and the three Bose forms;
* the on-shell detailed-balance identities of the Bose combinations;
* the classical limit rate(2T)/rate(T) -> 4;
* exact quadratic scaling in Phi4 and zero rates at Phi4 = 0;
* equal rates at symmetry-equivalent q for point-group-symmetric force constants;
* accepted-term counts from an independent vectorised enumeration of the window rule.
"""
import numpy as np
import pytest

import oracle
import oracle.brute as brute
import oracle.modes as om
from paper_2104_04895_gb300 import synth
from conftest import oracle_modes

HBAR_SI = 1.054571817e-34     # J s
KB_SI = 1.380649e-23          # J/K
EV = 1.602176634e-19
AMU_SI = 1.66053906660e-27
ANG = 1e-10


def bose_si(w_rad_ps, T):
    return 1.0 / np.expm1(HBAR_SI * w_rad_ps * 1e12 / (KB_SI * T))


def test_single_q_closed_form_in_si_units(rng):
    cr = synth.diamond_si((1, 1, 1))
    nb = cr.nb
    omega = np.array([[3.0, 1.0, 1.0, 1.0, 7.0, 11.0]])
    # random unitary eigenvectors (complex, so that the conjugated legs matter)
    A = rng.normal(size=(nb, nb)) + 1j * rng.normal(size=(nb, nb))
    Q, _ = np.linalg.qr(A)
    evec = Q.T[None, :, :].copy()
    vel = np.zeros((1, nb, 3))
    T = 300.0
    rates, acc = oracle.rates4(cr, omega, evec, vel, temps=[T], scalebroad=1.0)
    P = brute.supercell_phi4(cr)
    mult = {0: 0.5, 1: 0.5, 2: 1.0 / 6.0}
    signs = {0: (1, 1), 1: (1, -1), 2: (-1, -1)}
    # brute-force vertex in eV/(A^4 amu^2) -> SI J/(m^4 kg^2)
    vconv = EV / ANG**4 / AMU_SI**2
    n = bose_si(omega[0], T)
    count = np.zeros(3)
    for lam in range(nb):
        expect = 0.0
        for pr in range(3):
            s1, s2 = signs[pr]
            V = brute.vertex(cr, P, evec, 0, 0, 0, 0, conj1=s1 < 0, conj2=s2 < 0)
            for j1 in range(nb):
                for j2 in range(nb):
                    for j3 in range(nb):
                        dw = omega[0, lam] + s1 * omega[0, j1] + s2 * omega[0, j2] - omega[0, j3]
                        if dw != 0.0:
                            continue
                        count[pr] += 1
                        if pr == 0:
                            B = (1 + n[j1]) * (1 + n[j2]) * n[j3]
                        elif pr == 1:
                            B = (1 + n[j1]) * n[j2] * n[j3]
                        else:
                            B = n[j1] * n[j2] * n[j3]
                        wsi = omega[0, [lam, j1, j2, j3]] * 1e12
                        # Gamma_p = hbar^2 pi / (8N) B/n |V|^2 delta / prod(w); delta = 1 ps = 1e-12 s; N = 1
                        gam = HBAR_SI**2 * np.pi / 8.0 * B / n[lam] * abs(V[lam, j1, j2, j3] * vconv) ** 2 \
                            * 1e-12 / np.prod(wsi)
                        expect += mult[pr] * gam
        expect_ps = expect * 1e-12
        assert rates[0, lam] == pytest.approx(expect_ps, rel=1e-9, abs=1e-300), lam
    assert np.array_equal(acc, count)
    assert acc.min() > 0  # every process is exercised


def test_detailed_balance_on_shell():
    for T in (50.0, 300.0, 1000.0):
        for (w, w1, w2) in [(1.0, 2.0, 3.5), (10.0, 0.3, 7.0), (25.0, 20.0, 1.0)]:
            n = lambda x: oracle.bose(x, T)
            # ++ : w''' = w + w' + w''
            w3 = w + w1 + w2
            lhs = (1 + n(w1)) * (1 + n(w2)) * n(w3) / n(w)
            rhs = n(w1) * n(w2) * (1 + n(w3)) / (1 + n(w))
            assert lhs == pytest.approx(rhs, rel=1e-12)
            # +- : w + w' = w'' + w'''
            w3 = w + w1 - w2 if w + w1 - w2 > 0 else None
            if w3:
                lhs = (1 + n(w1)) * n(w2) * n(w3) / n(w)
                rhs = n(w1) * (1 + n(w2)) * (1 + n(w3)) / (1 + n(w))
                assert lhs == pytest.approx(rhs, rel=1e-12)
            # -- : w = w' + w'' + w'''
            W = w1 + w2 + 4.0
            lhs = n(w1) * n(w2) * n(4.0) / n(W)
            rhs = (1 + n(w1)) * (1 + n(w2)) * (1 + n(4.0)) / (1 + n(W))
            assert lhs == pytest.approx(rhs, rel=1e-12)
    # Bose values against the SI definition
    for w in (0.1, 5.0, 50.0):
        assert oracle.bose(w, 300.0) == pytest.approx(bose_si(w, 300.0), rel=1e-9)


def test_classical_limit_quadratic_in_T():
    cr = synth.simple_cubic((3, 3, 3))
    w, e, v = oracle_modes(cr)
    sel = [3 * 5 + 1, 3 * 13 + 2]
    r, _ = oracle.rates4(cr, w, e, v, temps=[1e6, 2e6], sel=sel)
    ratio = r[1] / r[0]
    np.testing.assert_allclose(ratio, 4.0, rtol=2e-3)


def test_quadratic_scaling_and_zero():
    cr = synth.simple_cubic((3, 3, 2))
    w, e, v = oracle_modes(cr)
    r1, a1 = oracle.rates4(cr, w, e, v)
    r2, a2 = oracle.rates4(cr.scaled_fc4(2.0), w, e, v)
    assert np.array_equal(r2, 4.0 * r1)
    assert np.array_equal(a1, a2)
    r0, a0 = oracle.rates4(cr.scaled_fc4(0.0), w, e, v)
    assert np.all(r0 == 0.0) and np.array_equal(a0, a1)
    assert r1.max() > 0


def _avg_degenerate(rates_row, omega_row):
    out = rates_row.copy()
    for (b, e_) in om.degenerate_sets(omega_row):
        out[b:e_] = rates_row[b:e_].mean()
    return out


def test_symmetry_equivalent_q_have_equal_rates():
    cr = synth.simple_cubic((4, 4, 4), symmetric=True)
    w, e, v = oracle_modes(cr)
    nb = cr.nb
    # grid points related by the cubic group: (1,0,0), (0,1,0), (0,0,3) and (1,2,0), (2,0,3)
    groups = [[(1, 0, 0), (0, 1, 0), (0, 0, 3), (3, 0, 0)], [(1, 2, 0), (2, 0, 3), (0, 3, 2)]]
    for grp in groups:
        qs = [(g[0] * 4 + g[1]) * 4 + g[2] for g in grp]
        sel = [q * nb + j for q in qs for j in range(nb)]
        r, _ = oracle.rates4(cr, w, e, v, sel=sel)
        rows = [_avg_degenerate(r[0, k * nb:(k + 1) * nb], w[qs[k]]) for k in range(len(qs))]
        for k in range(1, len(qs)):
            np.testing.assert_allclose(rows[k], rows[0], rtol=1e-9)


def test_accepted_counts_by_enumeration():
    cr = synth.simple_cubic((3, 3, 3))
    w, e, v = oracle_modes(cr)
    nb, N = cr.nb, cr.nq
    G = om.grid_points(cr.grid)
    ng = np.array(cr.grid)
    B = om.reciprocal(cr.lattice)
    dq = (abs(np.linalg.det(B)) / N) ** (1.0 / 3.0)
    sel = [nb * 4 + 1, nb * 10 + 2, nb * 22]
    _, acc = oracle.rates4(cr, w, e, v, sel=sel, window=2.0)
    count = np.zeros(3)
    for m in sel:
        q, j = divmod(m, nb)
        for pr, (s1, s2) in enumerate([(1, 1), (1, -1), (-1, -1)]):
            g3 = (G[q][None, None, :] + s1 * G[:, None, :] + s2 * G[None, :, :]) % ng
            q3 = (g3[..., 0] * ng[1] + g3[..., 1]) * ng[2] + g3[..., 2]          # (q1, q2)
            W1 = w[:, None, :, None, None]                                     # q1, -, j1
            W2 = w[None, :, None, :, None]                                     # -, q2, -, j2
            W3 = w[q3][:, :, None, None, :]                                    # q1, q2, -, -, j3
            t = (w[q, j] + s1 * W1) + s2 * W2
            dw = t - W3
            V2 = v[None, :, None, :, None, :]
            V3 = v[q3][:, :, None, None, :, :]
            d = V2 - V3
            sig = (1.0 * np.sqrt((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2])) * dq
            ok = (np.abs(dw) <= 2.0 * np.where(sig < 1e-10, 1e-10, sig)) & (W1 != 0) & (W2 != 0) & (W3 != 0)
            count[pr] += ok.sum()
    assert np.array_equal(acc, count)


def test_process_classes_split_the_rate():
    """Eq. 4phgamma sums three process classes; the oracle's per-class rates add up to the full rate, and
    each class carries exactly its own accepted terms (whose totals the enumeration above pins)."""
    cr = synth.simple_cubic((3, 3, 3))
    w, e, v = oracle_modes(cr)
    nb = cr.nb
    sel = [nb * 4 + 1, nb * 10 + 2, nb * 22, nb * 13]
    temps = [150.0, 600.0]
    full, acc = oracle.rates4(cr, w, e, v, sel=sel, temps=temps)
    parts = []
    for p in range(3):
        r, a = oracle.rates4(cr, w, e, v, sel=sel, temps=temps, processes=(p,))
        expect = np.zeros(3)
        expect[p] = acc[p]
        assert np.array_equal(a, expect)
        assert np.all(r >= 0.0)
        parts.append(r)
    assert acc[0] > 0 and acc[1] > 0 and acc[2] > 0
    np.testing.assert_allclose(parts[0] + parts[1] + parts[2], full, rtol=1e-13, atol=0.0)
    two, _ = oracle.rates4(cr, w, e, v, sel=sel, temps=temps, processes=(0, 2))
    np.testing.assert_allclose(two, parts[0] + parts[2], rtol=1e-13, atol=0.0)


def test_umklapp_hand_worked_cases():
    """Normal/Umklapp (Sec. 2.2: q''' = q + s1 q' + s2 q'' + Q, Q = 0 normal) with each wavevector taken as its
    shortest translate, ties to the smallest shift. Cases worked by hand on simple-cubic grids."""
    idx = lambda g, n: (g[0] * n + g[1]) * n + g[2]
    cr3 = synth.simple_cubic((3, 3, 3))  # representatives 0, 1/3, -1/3 (no ties)
    x1, x2, G = idx((1, 0, 0), 3), idx((2, 0, 0), 3), 0
    # ++: 1/3 + 1/3 + 1/3 = 1 -> q''' = Gamma, Q = 1: Umklapp
    assert oracle.umklapp(cr3, x1, x1, x1, 0) == 1
    # ++: 1/3 + 1/3 + 0 = 2/3 ~ -1/3: Umklapp
    assert oracle.umklapp(cr3, x1, x1, G, 0) == 1
    # ++: 1/3 + (-1/3) + 0 = 0: normal
    assert oracle.umklapp(cr3, x1, x2, G, 0) == 0
    # +-: 1/3 + 1/3 - 1/3 = 1/3: normal
    assert oracle.umklapp(cr3, x1, x1, x1, 1) == 0
    # --: 1/3 - (-1/3) - (-1/3) = 1 ~ 0: Umklapp
    assert oracle.umklapp(cr3, x1, x2, x2, 2) == 1
    # --: 1/3 - 1/3 - 0 = 0: normal
    assert oracle.umklapp(cr3, x1, x1, G, 2) == 0
    cr2 = synth.simple_cubic((2, 2, 2))  # 1/2 and -1/2 tie: the representative is +1/2
    y = idx((1, 0, 0), 2)
    assert oracle.umklapp(cr2, y, y, y, 0) == 1      # 3/2 - 1/2 = 1
    assert oracle.umklapp(cr2, y, y, y, 1) == 0      # 1/2 + 1/2 - 1/2 - 1/2 = 0
    assert oracle.umklapp(cr2, G, G, y, 0) == 0      # 0 + 0 + 1/2 - 1/2 = 0
    d = idx((1, 1, 0), 2)                            # (1/2, 1/2, 0): four tied translates, (+1/2, +1/2, 0) wins
    assert oracle.umklapp(cr2, d, y, G, 1) == 1      # (1/2, 1/2, 0) + (1/2, 0, 0) - 0 - (0, 1/2, 0) = (1, 0, 0)
    assert oracle.umklapp(cr2, d, G, G, 1) == 0      # q''' = q
    cr4 = synth.simple_cubic((4, 4, 4))  # 1/4, -1/4 and the tie 1/2 = -1/2 together: the tie rule decides
    h, f, f3 = idx((2, 0, 0), 4), idx((1, 0, 0), 4), idx((3, 0, 0), 4)
    G4 = 0
    assert oracle.umklapp(cr4, h, f, G4, 0) == 1     # 1/2 + 1/4 + 0 - (-1/4) = 1 (with -1/2 it would be 0)
    assert oracle.umklapp(cr4, f, f, G4, 0) == 0     # 1/4 + 1/4 + 0 - 1/2 = 0 (with -1/2 it would be 1)
    assert oracle.umklapp(cr4, f3, f3, G4, 0) == 1   # -1/4 - 1/4 + 0 - 1/2 = -1
    assert oracle.umklapp(cr4, h, f3, G4, 1) == 0    # 1/2 - 1/4 - 0 - 1/4 = 0


def test_normal_and_umklapp_split_the_rate():
    """The normal and Umklapp parts add up to the full rate, per process class, with the counts split alike;
    on a 1 x 1 x 1 grid every wavevector is Gamma and every process is normal."""
    cr = synth.diamond_si((3, 3, 2))
    w, e, v = oracle_modes(cr)
    nb = cr.nb
    sel = [nb * 1 + 2, nb * 7 + 4, nb * 12 + 5]
    full, acc = oracle.rates4(cr, w, e, v, sel=sel)
    rn, an = oracle.rates4(cr, w, e, v, sel=sel, nu="normal")
    ru, au = oracle.rates4(cr, w, e, v, sel=sel, nu="umklapp")
    assert np.array_equal(an + au, acc) and an[1] > 0 and au[1] > 0
    np.testing.assert_allclose(rn + ru, full, rtol=1e-13, atol=0.0)
    one = synth.diamond_si((1, 1, 1))
    w1, e1, v1 = oracle_modes(one)
    f1, a1 = oracle.rates4(one, w1, e1, v1)
    n1, b1 = oracle.rates4(one, w1, e1, v1, nu="normal")
    u1, c1 = oracle.rates4(one, w1, e1, v1, nu="umklapp")
    assert np.array_equal(n1, f1) and np.array_equal(b1, a1)
    assert np.all(u1 == 0.0) and np.all(c1 == 0.0)


def test_umklapp_classification_is_point_group_invariant(rng):
    """On an odd simple-cubic grid no wavevector lies on the zone boundary, so the shortest translates are unique
    and the normal/Umklapp split must be invariant under the 48 cubic operations applied to all partners."""
    cr = synth.simple_cubic((3, 3, 3), symmetric=True)
    ops = synth.point_group_ops(cr)
    n = 3
    idx = lambda g: int(((g[0] % n) * n + g[1] % n) * n + g[2] % n)
    G = np.array(np.unravel_index(np.arange(cr.nq), cr.grid)).T
    seen = set()
    for _ in range(30):
        q, q1, q2 = (int(x) for x in rng.integers(0, cr.nq, size=3))
        for pr in range(3):
            u = oracle.umklapp(cr, q, q1, q2, pr)
            seen.add(u)
            for R in ops[::5]:
                assert oracle.umklapp(cr, idx(R @ G[q]), idx(R @ G[q1]), idx(R @ G[q2]), pr) == u
    assert seen == {0, 1}


def test_umklapp_reading_on_a_sheared_cell(rng):
    """On a strongly sheared cell the shortest translate of some grid wavevectors needs a shift of 2 reciprocal
    vectors.  The classification must follow the reading exactly: a brute-force search written here (shortest
    sum_a (g_a / N_a - m_a) b_a over m_a in [-2, 2], ties to the lexicographically smallest m) gives every
    representative, and Q = 0 decides normal against Umklapp for every process of the grid."""
    import itertools
    a = 3.0
    lattice = a * np.array([[1.0, -5.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    cr = synth.simple_cubic((4, 4, 2)).with_grid((4, 4, 2))
    cr.lattice = lattice
    grid = np.array(cr.grid)
    B = 2.0 * np.pi * np.linalg.inv(lattice).T
    shifts = sorted(itertools.product(range(-2, 3), repeat=3))      # lexicographic order
    G = np.array(np.unravel_index(np.arange(cr.nq), cr.grid)).T
    rep = np.zeros((cr.nq, 3))
    need2 = 0
    for q in range(cr.nq):
        best, bm = None, None
        for m in shifts:
            k = (G[q] / grid - np.array(m)) @ B
            l2 = float(k @ k)
            if best is None or l2 < best * (1.0 - 1e-9):
                best, bm = l2, m
        rep[q] = G[q] / grid - np.array(bm)                          # reduced coordinates of the representative
        need2 += max(abs(x) for x in bm) == 2
    assert need2 > 0                                                 # the cell exercises shifts of 2
    idx = lambda g: int(((g[0] % grid[0]) * grid[1] + g[1] % grid[1]) * grid[2] + g[2] % grid[2])
    signs = {0: (1, 1), 1: (1, -1), 2: (-1, -1)}
    seen = set()
    for _ in range(400):
        q, q1, q2 = (int(x) for x in rng.integers(0, cr.nq, size=3))
        for pr, (s1, s2) in signs.items():
            q3 = idx(G[q] + s1 * G[q1] + s2 * G[q2])
            Q = rep[q] + s1 * rep[q1] + s2 * rep[q2] - rep[q3]
            expect = int(np.abs(Q).max() > 1e-9)
            assert oracle.umklapp(cr, q, q1, q2, pr) == expect, (q, q1, q2, pr)
            seen.add(expect)
    assert seen == {0, 1}
