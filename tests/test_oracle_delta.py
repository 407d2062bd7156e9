"""Pins of the oracle's finite-sigma Gaussian (Sec. 2.4 and App. B) and of time reversal.

The energy delta of Eq. 4phgamma is a Gaussian of width sigma = scalebroad |v'' - v'''| |dq| (Sec. 2.4,
the final broadening of App. B), delta = exp(-dw^2/sigma^2) / (sqrt(pi) sigma).  These tests fix it
by mathematics rather than by restating the oracle's expression:

* a single-q crystal (1x1x1 grid) whose injected frequencies put exactly one family of ++ terms near
  energy conservation while the injected mode frequency of their third partner is swept by s, so that
  every accepted term has dw = -s and the same sigma; the extracted delta(s), integrated over s by a
  midpoint sum, must give erf(window) (the mass of a normalised Gaussian inside |s| <= window sigma),
  whatever sigma is; its peak must be 1/(sqrt(pi) sigma) and its support must end at |s| = window sigma
  with sigma worked out by hand from the lattice and the injected velocities -- for the isotropic
  |dq| = (|det B|/N)^(1/3) and for the per-axis form on an orthorhombic cell;
* a single-q SI-unit closed form with finite sigma: the rate of every mode is rebuilt term by term from
  the supercell brute-force vertex with the Gaussian evaluated in SI units (rad/s, m/s, 1/m);
* time reversal: with real force constants and e(-q) = conj e(q), V(-q; -q', -q'') = conj V(q; q', q'')
  and each mode's rate at -q equals its rate at q, for force constants without point-group symmetry.

The unit-vertex option (|V|^2 := 1, no prefactor) isolates the delta in the first group.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_2104_04895_gb300 import synth
from conftest import oracle_modes

HBAR_SI = 1.054571817e-34     # J s
KB_SI = 1.380649e-23          # J/K
EV = 1.602176634e-19
AMU_SI = 1.66053906660e-27
ANG = 1e-10
WINDOW = 2.0
T = 300.0


def bose_si(w_rad_ps, temp):
    return 1.0 / np.expm1(HBAR_SI * w_rad_ps * 1e12 / (KB_SI * temp))


def grid_crystal(lattice, grid):
    """Simple-cubic force constants (only their presence matters under the unit vertex) on the given grid, with
    the given lattice rows (A)."""
    cr = synth.simple_cubic(grid)
    cr.lattice = np.asarray(lattice, dtype=np.float64)
    return cr


def hand_sigma(lattice, grid, dv, sb, dq_mode):
    """sigma = sb |dv| |dq| with |dq| = (|det B| / N)^(1/3), or the per-axis form sb sqrt(sum_a ((dv.b_a)/N_a)^2/3),
    for an orthorhombic cell (b_a = 2 pi / a_a along axis a), worked out from the axis lengths and the grid."""
    a = np.diag(lattice)
    assert np.allclose(lattice, np.diag(a))
    if dq_mode == 0:
        detB = (2 * math.pi) ** 3 / (a[0] * a[1] * a[2])
        return sb * math.sqrt(sum(x * x for x in dv)) * (detB / (grid[0] * grid[1] * grid[2])) ** (1.0 / 3.0)
    comps = [dv[k] * 2 * math.pi / a[k] / grid[k] for k in range(3)]
    return sb * math.sqrt(sum(c * c for c in comps) / 3.0)


def swept_delta(cr, s_values, sb, dq_mode, va, vb):
    """delta(s) extracted from the unit-vertex ++ rate of mode (q = 0, j = 0) with omega(q = 0) = (1, 1, 3 + s)
    and omega = (50, 60, 70) at every other grid point.

    ++ terms of that mode (omega = 1): dw = ((1 + w1) + w2) - w3.  With both partners at Gamma (so the third is
    at Gamma too), j1, j2 in {0, 1} and j3 = 2 it is -s and sigma = sb |v(0 or 1) - v(2)| |dq|; every other ++
    term misses energy conservation by 2 or more, outside the window for the sigma used here.  Each of the four
    accepted terms carries 1/2 (1 + n1)(1 + n2) n3 / n0 / (w w1 w2 w3) (Eq. 4phgamma with |V|^2 := 1), computed
    here with the oracle's Bose factor (pinned against the SI definition elsewhere, and taken from it so that the
    truncated constants do not blur the delta), and the rate divided by their sum is delta(s).
    """
    N = cr.nq
    evec = np.tile(np.eye(3, dtype=complex)[None], (N, 1, 1))
    vel = np.zeros((N, 3, 3))
    vel[0] = [va, va, vb]
    out = []
    for s in s_values:
        omega = np.tile(np.array([[50.0, 60.0, 70.0]]), (N, 1))
        omega[0] = [1.0, 1.0, 3.0 + s]
        r, acc = oracle.rates4(cr, omega, evec, vel, temps=[T], scalebroad=sb, window=WINDOW, dq_mode=dq_mode,
                               sel=[0], unit_vertex=True, processes=(0,))
        n = np.array([oracle.bose(x, T) for x in omega[0]])
        weight = 4 * 0.5 * (1 + n[0]) * (1 + n[0]) * n[2] / n[0] / (omega[0, 0] ** 3 * omega[0, 2])
        assert acc[0] in (0.0, 4.0) and acc[1] == 0.0 and acc[2] == 0.0
        out.append(r[0, 0] / weight)
    return np.array(out)


GEOMETRIES = [
    # (lattice rows, grid, v(0) = v(1), v(2), scalebroad, dq_mode)
    (np.diag([3.0, 4.0, 5.0]), (2, 3, 1), (0.3, -0.2, 0.5), (0.0, 0.1, -0.1), 0.7, 0),
    (np.diag([3.0, 4.0, 5.0]), (2, 3, 1), (0.3, -0.2, 0.5), (0.0, 0.1, -0.1), 0.7, 1),
    (np.diag([2.5, 2.5, 6.0]), (1, 1, 1), (1.1, 0.0, 0.0), (0.0, 0.0, 0.4), 0.2, 1),
]


@pytest.mark.parametrize("lattice,grid,va,vb,sb,dq_mode", GEOMETRIES,
                         ids=["iso-2x3x1", "per-axis-2x3x1", "per-axis-tetragonal-1x1x1"])
def test_gaussian_is_normalised_and_its_width_is_the_hand_sigma(lattice, grid, va, vb, sb, dq_mode):
    cr = grid_crystal(lattice, grid)
    dv = [va[k] - vb[k] for k in range(3)]
    sig = hand_sigma(lattice, grid, dv, sb, dq_mode)
    assert 0.05 < sig < 0.9  # window edge well inside the gap of 2 to the other terms, sigma far from 1
    # peak and shape: delta(0) = 1/(sqrt(pi) sigma); delta(sigma)/delta(0) = e^-1; delta(1.5 sigma)/delta(0) = e^-2.25
    d = swept_delta(cr, [0.0, sig, -1.5 * sig], sb, dq_mode, va, vb)
    assert d[0] == pytest.approx(1.0 / (math.sqrt(math.pi) * sig), rel=1e-12)
    assert d[1] / d[0] == pytest.approx(math.exp(-1.0), rel=1e-9)
    assert d[2] / d[0] == pytest.approx(math.exp(-2.25), rel=1e-9)
    # support: the window |dw| <= 2 sigma
    edge = swept_delta(cr, [WINDOW * sig * (1 - 1e-7), -WINDOW * sig * (1 - 1e-7), WINDOW * sig * (1 + 1e-7),
                            -WINDOW * sig * (1 + 1e-7)], sb, dq_mode, va, vb)
    assert edge[0] > 0 and edge[1] > 0 and edge[2] == 0.0 and edge[3] == 0.0
    # normalisation: the midpoint sum of delta over s tends to erf(window)
    n = 1000
    h = 2.2 * WINDOW * sig / n
    s = -1.1 * WINDOW * sig + h * (np.arange(n) + 0.5)
    mass = float(np.sum(swept_delta(cr, s, sb, dq_mode, va, vb)) * h)
    assert mass == pytest.approx(math.erf(WINDOW), abs=2e-4)


def test_small_sigma_rule_gives_unit_delta():
    """Velocities equal on both legs: sigma = 0 < sigma_min, so delta := 1 (Sec. 2.4) inside the window
    |dw| <= window * sigma_min and 0 outside it."""
    cr = grid_crystal(np.diag([3.0, 3.0, 3.0]), (1, 1, 1))
    v = (0.2, 0.1, -0.3)
    d = swept_delta(cr, [0.0, 1e-11, 3e-10], 1.0, 0, v, v)
    assert d[0] == pytest.approx(1.0, rel=1e-13) and d[1] == pytest.approx(1.0, rel=1e-13) and d[2] == 0.0


def test_single_q_si_closed_form_with_finite_sigma(rng):
    """Rates of a 1x1x1 diamond crystal with injected frequencies close to (not at) energy conservation and
    injected velocities, rebuilt term by term in SI units from the supercell brute-force vertex: Gamma_p =
    hbar^2 pi / (8N) B_p / n |V|^2 delta / prod(w) with delta = exp(-dw^2/sigma^2)/(sqrt(pi) sigma) in seconds,
    sigma = sb |v'' - v'''| |dq| in rad/s, and the window |dw| <= 2 max(sigma, sigma_min)."""
    cr = synth.diamond_si((1, 1, 1))
    nb = cr.nb
    omega = np.array([[3.0, 1.004, 0.997, 1.0, 7.01, 10.995]])
    A = rng.normal(size=(nb, nb)) + 1j * rng.normal(size=(nb, nb))
    Q, _ = np.linalg.qr(A)
    evec = Q.T[None, :, :].copy()
    vel = rng.normal(scale=0.02, size=(1, nb, 3))
    sb = 1.0
    rates, acc = oracle.rates4(cr, omega, evec, vel, temps=[T], scalebroad=sb)
    P = brute.supercell_phi4(cr)
    mult = {0: 0.5, 1: 0.5, 2: 1.0 / 6.0}
    signs = {0: (1, 1), 1: (1, -1), 2: (-1, -1)}
    vconv = EV / ANG**4 / AMU_SI**2                    # eV/(A^4 amu^2) -> J/(m^4 kg^2)
    Bm = 2 * np.pi * np.linalg.inv(cr.lattice).T / ANG   # reciprocal vectors in 1/m
    dq_si = abs(np.linalg.det(Bm)) ** (1.0 / 3.0)       # N = 1
    vel_si = vel * ANG / 1e-12                          # A/ps -> m/s
    sigmin_si = 1e-10 * 1e12
    n = bose_si(omega[0], T)
    count = np.zeros(3)
    finite = 0
    for lam in range(nb):
        expect = 0.0
        for pr in range(3):
            s1, s2 = signs[pr]
            V = brute.vertex(cr, P, evec, 0, 0, 0, 0, conj1=s1 < 0, conj2=s2 < 0)
            for j1 in range(nb):
                for j2 in range(nb):
                    for j3 in range(nb):
                        w = omega[0, [lam, j1, j2, j3]] * 1e12      # rad/s
                        dw = w[0] + s1 * w[1] + s2 * w[2] - w[3]
                        sig = sb * np.linalg.norm(vel_si[0, j2] - vel_si[0, j3]) * dq_si
                        if abs(dw) > WINDOW * max(sig, sigmin_si) * (1 + 1e-9):
                            continue
                        assert abs(dw) < WINDOW * max(sig, sigmin_si) * (1 - 1e-6)  # no case at the edge
                        count[pr] += 1
                        if sig < sigmin_si:
                            delta = 1e-12                            # delta := 1 ps
                        else:
                            delta = np.exp(-(dw / sig) ** 2) / (np.sqrt(np.pi) * sig)
                            finite += 1
                        if pr == 0:
                            B = (1 + n[j1]) * (1 + n[j2]) * n[j3]
                        elif pr == 1:
                            B = (1 + n[j1]) * n[j2] * n[j3]
                        else:
                            B = n[j1] * n[j2] * n[j3]
                        gam = HBAR_SI**2 * np.pi / 8.0 * B / n[lam] * abs(V[lam, j1, j2, j3] * vconv) ** 2 \
                            * delta / np.prod(w)
                        expect += mult[pr] * gam
        assert rates[0, lam] == pytest.approx(expect * 1e-12, rel=1e-9, abs=1e-300), lam
    assert np.array_equal(acc, count)
    assert finite >= 10  # the finite-sigma Gaussian carries a real share of the terms


def test_vertex_under_time_reversal():
    """V(-q; -q', -q'') = conj V(q; q', q'') for real Phi4 with e(-q) = conj e(q) (Eq. V4), per process."""
    cr = synth.diamond_si((3, 3, 2))
    _, e, _ = oracle_modes(cr)
    n = cr.grid

    def neg(q):
        g = np.unravel_index(q, n)
        return int(np.ravel_multi_index(tuple((-np.asarray(g)) % np.asarray(n)), n))

    for (q, q1, q2) in [(1, 4, 7), (5, 11, 2), (13, 0, 17)]:
        for pr in range(3):
            V, q3 = oracle.v4(cr, e, q, q1, q2, pr)
            Vm, q3m = oracle.v4(cr, e, neg(q), neg(q1), neg(q2), pr)
            assert q3m == neg(q3)
            assert np.abs(V).max() > 0
            np.testing.assert_allclose(Vm, np.conj(V), rtol=0, atol=1e-12 * np.abs(V).max())


@pytest.mark.parametrize("maker", [lambda: synth.diamond_si((3, 3, 2)), lambda: synth.zincblende_bas((3, 2, 2))],
                         ids=["diamond-3x3x2", "bas-3x2x2"])
def test_rates_are_even_in_q_per_mode(maker):
    """rate(-q, j) = rate(q, j) for every branch, with per-bond random Phi4 (no point-group symmetry), two
    temperatures and dq_mode 1 as well: the terms at -q are those at q with all wavevectors negated, with
    equal frequencies, |V|^2 and sigma, so the window accepts the same number of terms."""
    cr = maker()
    w, e, v = oracle_modes(cr)
    nb, n = cr.nb, cr.grid
    pairs = []
    for q in range(cr.nq):
        g = np.unravel_index(q, n)
        m = int(np.ravel_multi_index(tuple((-np.asarray(g)) % np.asarray(n)), n))
        if m > q:
            pairs.append((q, m))
    assert len(pairs) >= 3
    for dq_mode in (0, 1):
        for (q, m) in pairs[:3]:
            ra, aa = oracle.rates4(cr, w, e, v, temps=[200.0, 900.0], dq_mode=dq_mode, sel=[q * nb + j for j in range(nb)])
            rb, ab = oracle.rates4(cr, w, e, v, temps=[200.0, 900.0], dq_mode=dq_mode, sel=[m * nb + j for j in range(nb)])
            assert np.array_equal(aa, ab) and aa.sum() > 0
            np.testing.assert_allclose(rb, ra, rtol=1e-13, atol=0.0)


def test_rates_are_intensive():
    """The outer 1/N of Eq. tao0 and the 1/N of Gamma (Eq. 4phgamma) make the rate intensive.  With on-site
    quartets only (all cell vectors 0) every phase of Eq. V4 is 1, so with the same injected modes at every grid
    point each of the N^2 (q', q'') pairs repeats the single-q sum: the rates on a 2x3x1 grid must equal those on
    a 1x1x1 grid.  Integer frequencies and zero velocities make delta := 1 on exactly conserving terms."""
    base = synth.simple_cubic((1, 1, 1))
    onsite = np.all(base.fc4_idx[:, 4:13] == 0, axis=1)
    assert onsite.sum() >= 1
    rng = np.random.Generator(np.random.PCG64(5))
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    rates = []
    for grid in ((1, 1, 1), (2, 3, 1)):
        cr = base.with_grid(grid)
        cr.fc4_idx = base.fc4_idx[onsite]
        cr.fc4_val = base.fc4_val[onsite]
        N = cr.nq
        omega = np.tile(np.array([[1.0, 2.0, 3.0]]), (N, 1))
        evec = np.tile(Q.T[None].astype(complex), (N, 1, 1))
        r, acc = oracle.rates4(cr, omega, evec, np.zeros((N, 3, 3)), temps=[300.0], sel=[0, 1, 2])
        assert acc.sum() > 0
        rates.append(r)
    assert rates[0].min() > 0
    np.testing.assert_allclose(rates[1], rates[0], rtol=1e-12, atol=0.0)


def test_phase_space_p4_single_q_closed_form():
    """The unweighted phase space (BTE.P4 of Appendix A, the rate's sum with the vertex, Bose and frequency factors
    set to 1): with zero velocities and integer frequencies only exactly conserving terms enter, each with delta := 1,
    so P4 of each mode is 1/2 n++ + 1/2 n+- + 1/6 n-- with n_p its accepted counts (pinned by enumeration)."""
    cr = synth.diamond_si((1, 1, 1))
    omega = np.array([[3.0, 1.0, 1.0, 2.0, 4.0, 6.0]])
    evec = np.eye(6, dtype=complex)[None]
    vel = np.zeros((1, 6, 3))
    for lam in range(6):
        p4, acc = oracle.rates4(cr, omega, evec, vel, temps=[T], sel=[lam], unit_vertex=2)
        assert p4[0, 0] == pytest.approx(0.5 * acc[0] + 0.5 * acc[1] + acc[2] / 6.0, rel=1e-13, abs=0)
        if lam == 0:
            assert acc.min() > 0


def test_phase_space_p4_is_the_swept_gaussian():
    """With the unit weights the swept family of test_gaussian... contributes 4 * 1/2 * delta(s): the P4 sum over the
    sweep is 2 erf(window) times the step, whatever sigma is."""
    lattice, grid, va, vb, sb, dq_mode = GEOMETRIES[0]
    cr = grid_crystal(lattice, grid)
    N = cr.nq
    sig = hand_sigma(lattice, grid, [va[k] - vb[k] for k in range(3)], sb, dq_mode)
    evec = np.tile(np.eye(3, dtype=complex)[None], (N, 1, 1))
    vel = np.zeros((N, 3, 3))
    vel[0] = [va, va, vb]
    n = 600
    h = 2.2 * WINDOW * sig / n
    total = 0.0
    for s in -1.1 * WINDOW * sig + h * (np.arange(n) + 0.5):
        omega = np.tile(np.array([[50.0, 60.0, 70.0]]), (N, 1))
        omega[0] = [1.0, 1.0, 3.0 + s]
        r, _ = oracle.rates4(cr, omega, evec, vel, temps=[T], scalebroad=sb, sel=[0], unit_vertex=2, processes=(0,))
        total += r[0, 0] * h
    assert total == pytest.approx(2.0 * math.erf(WINDOW), abs=5e-4)
