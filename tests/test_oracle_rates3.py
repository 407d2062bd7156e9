"""Pins of the oracle's three-phonon rates (Eqs. tao0, 3phgamma, V3).

* brute force: the Born-von Karman supercell sum over every atom triplet equals Eq. V3 on tiny grids, for
  both processes (e^{-lambda'} = conj e(lambda'));
* the vertex is symmetric under exchanging its last two legs with time reversal: V+(q, q', q'') equals
  V-(q, -q', q'') for the same triple of modes;
* |V|^2 := 1 turns the rate sum into the weighted three-phonon phase space that oracle.phase3 computes
  independently; the rates are exactly quadratic in Phi3 and vanish with it.
"""
import numpy as np
import pytest

import oracle
import oracle.brute as brute
import oracle.modes as om
from paper_2104_04895_gb300 import synth
from conftest import oracle_modes


def idx_of(cr, g):
    ng = np.array(cr.grid)
    g = np.asarray(g) % ng
    return int((g[0] * ng[1] + g[1]) * ng[2] + g[2])


@pytest.mark.parametrize("maker", [lambda: synth.simple_cubic((2, 2, 2)), lambda: synth.simple_cubic((3, 2, 1)),
                                   lambda: synth.diamond_si((2, 1, 1)), lambda: synth.zincblende_bas((2, 2, 1))])
def test_vertex3_equals_supercell_brute_force(maker, rng):
    cr = maker()
    w, e, v = oracle_modes(cr)
    P3 = brute.supercell_phi3(cr)
    G = om.grid_points(cr.grid)
    natural = np.abs(cr.fc3_val).sum() / cr.mass.min() ** 1.5
    for trial in range(4):
        q, q1 = (int(x) for x in rng.integers(0, cr.nq, size=2))
        for pr, s1 in ((0, 1), (1, -1)):
            V, q2 = oracle.v3(cr, e, q, q1, pr)
            assert q2 == idx_of(cr, G[q] + s1 * G[q1])
            Vb = brute.vertex3(cr, P3, e, q, q1, q2, conj1=s1 < 0)
            scale = max(np.abs(Vb).max(), 1e-3 * natural)
            assert np.abs(V - Vb).max() <= 1e-12 * scale, (q, q1, pr)


def test_plus_and_minus_share_the_vertex():
    """V-(q, q') with q'' = q - q' equals V+(q, -q') (same q''), since e(-q') = conj e(q')."""
    cr = synth.diamond_si((3, 2, 2))
    w, e, v = oracle_modes(cr)
    G = om.grid_points(cr.grid)
    for q, q1 in ((1, 5), (7, 3), (0, 11)):
        Vm, q2m = oracle.v3(cr, e, q, q1, 1)
        Vp, q2p = oracle.v3(cr, e, q, idx_of(cr, -G[q1]), 0)
        assert q2m == q2p
        np.testing.assert_allclose(Vm, Vp, rtol=0, atol=1e-12 * np.abs(Vp).max())


def test_unit_vertex_is_the_weighted_phase_space():
    cr = synth.diamond_si((3, 3, 2))
    w, e, v = oracle_modes(cr)
    temps = [300.0, 800.0]
    sel = np.arange(cr.nb, cr.nq * cr.nb, 7)
    r1, acc = oracle.rates3(cr, w, e, v, temps=temps, sel=sel, unit_vertex=True)
    _, wp3 = oracle.phase3(cr, w, v, temps=temps, sel=sel)
    np.testing.assert_allclose(r1, wp3, rtol=1e-12, atol=0.0)
    assert acc[0] > 0 and acc[1] > 0


def test_quadratic_in_phi3():
    cr = synth.simple_cubic((3, 3, 3))
    w, e, v = oracle_modes(cr)
    sel = [5, 17, 40]
    r, _ = oracle.rates3(cr, w, e, v, sel=sel)
    c2 = cr.with_grid(cr.grid)
    c2.fc3_val = 2.0 * cr.fc3_val
    r2, _ = oracle.rates3(c2, w, e, v, sel=sel)
    assert np.array_equal(r2, 4.0 * r)
    c0 = cr.with_grid(cr.grid)
    c0.fc3_val = 0.0 * cr.fc3_val
    r0, _ = oracle.rates3(c0, w, e, v, sel=sel)
    assert np.all(r0 == 0.0) and np.all(r > 0.0)


HBAR_SI = 1.054571817e-34     # J s
KB_SI = 1.380649e-23          # J/K
EV = 1.602176634e-19
AMU_SI = 1.66053906660e-27
ANG = 1e-10


def test_single_q_closed_form_in_si_units(rng):
    """One q-point (1x1x1 grid), injected integer frequencies, v = 0: only exactly energy-conserving terms
    enter, each with delta := 1 ps. The rate then follows from Eqs. tao0 and 3phgamma written out in SI
    units with the brute-force supercell vertex, which pins the prefactor hbar pi / 4, the multiplicities
    1 and 1/2, the two Bose forms and the unit conversion term by term."""
    cr = synth.diamond_si((1, 1, 1))
    nb = cr.nb
    omega = np.array([[1.0, 2.0, 3.0, 3.0, 5.0, 8.0]])
    A = rng.normal(size=(nb, nb)) + 1j * rng.normal(size=(nb, nb))
    Q, _ = np.linalg.qr(A)
    evec = Q.T[None, :, :].copy()
    vel = np.zeros((1, nb, 3))
    T = 300.0
    rates, acc = oracle.rates3(cr, omega, evec, vel, temps=[T], scalebroad=1.0)
    P3 = brute.supercell_phi3(cr)
    vconv = EV / ANG**3 / AMU_SI**1.5          # eV/(A^3 amu^1.5) -> J/(m^3 kg^1.5)
    n = 1.0 / np.expm1(HBAR_SI * omega[0] * 1e12 / (KB_SI * T))
    count = np.zeros(2)
    for lam in range(nb):
        expect = 0.0
        for pr, s1 in ((0, 1), (1, -1)):
            V = brute.vertex3(cr, P3, evec, 0, 0, 0, conj1=s1 < 0)
            for j1 in range(nb):
                for j2 in range(nb):
                    if omega[0, lam] + s1 * omega[0, j1] - omega[0, j2] != 0.0:
                        continue
                    count[pr] += 1
                    B = (n[j1] - n[j2]) if pr == 0 else (n[j1] + n[j2] + 1.0)
                    wsi = omega[0, [lam, j1, j2]] * 1e12
                    # Gamma = hbar pi / 4 B |V|^2 delta / (w w' w''); delta = 1 ps; 1/N = 1; the - sum has 1/2
                    gam = HBAR_SI * np.pi / 4.0 * B * abs(V[lam, j1, j2] * vconv) ** 2 * 1e-12 / np.prod(wsi)
                    expect += (1.0 if pr == 0 else 0.5) * gam
        assert rates[0, lam] == pytest.approx(expect * 1e-12, rel=1e-9, abs=1e-300), lam
    assert np.array_equal(acc, count) and acc.min() > 0


def swept_delta3(cr, s_values, sb, dq_mode, va, vb, which):
    """delta(s) of the three-phonon paths, extracted on a crystal whose mode (q = 0, j = 0) has omega = 1, with
    omega(q = 0) = (1, 1, 2 + s) and omega = (50, 60, 70) at every other grid point.

    (+) terms of that mode: dw = (1 + w') - w''.  With q' = q'' = 0, j' in {0, 1} and j'' = 2 it is -s and sigma =
    sb |v(0 or 1) - v(2)| |dq|; every other term misses energy conservation by 1 or more, outside the window for the
    sigma used here.  which = "p3": P3 = (1/N) sum [delta+ + 1/2 delta-] holds 2 delta / N; which = "rates3": the
    unit-vertex three-phonon sum (1/N) sum B+ delta / (w w' w'') with B+ = n' - n'' holds 2 (n(1) - n(2 + s))
    delta / (N (2 + s)), with the oracle's Bose factor (pinned against the SI definition elsewhere)."""
    N = cr.nq
    evec = np.tile(np.eye(3, dtype=complex)[None], (N, 1, 1))
    vel = np.zeros((N, 3, 3))
    vel[0] = [va, va, vb]
    T = 300.0
    out = []
    for s in s_values:
        omega = np.tile(np.array([[50.0, 60.0, 70.0]]), (N, 1))
        omega[0] = [1.0, 1.0, 2.0 + s]
        if which == "p3":
            p3, _ = oracle.phase3(cr, omega, vel, temps=[T], scalebroad=sb, window=2.0, dq_mode=dq_mode, sel=[0])
            out.append(p3[0] * N / 2.0)
        else:
            r, acc = oracle.rates3(cr, omega, evec, vel, temps=[T], scalebroad=sb, window=2.0, dq_mode=dq_mode,
                                   sel=[0], unit_vertex=True)
            assert acc[0] in (0.0, 2.0) and acc[1] == 0.0
            weight = 2.0 * (oracle.bose(1.0, T) - oracle.bose(2.0 + s, T)) / (2.0 + s)
            out.append(r[0, 0] * N / weight)
    return np.array(out)


@pytest.mark.parametrize("which", ["p3", "rates3"])
@pytest.mark.parametrize("dq_mode", [0, 1])
def test_three_phonon_gaussian_is_normalised_and_its_width_is_the_hand_sigma(which, dq_mode):
    """The Gaussian of the three-phonon paths (Eq. 3phgamma with the broadening of Sec. 2.4 at the two partners),
    fixed by mathematics as for the four-phonon rates: peak 1/(sqrt(pi) sigma), e^-1 at s = sigma, support ending at
    window sigma, and a midpoint sum over s equal to erf(window), the mass of a normalised Gaussian; sigma worked
    out by hand from the orthorhombic cell, the grid and the injected velocities."""
    from test_oracle_delta import grid_crystal, hand_sigma
    lattice, grid = np.diag([3.0, 4.0, 5.0]), (2, 3, 1)
    va, vb, sb = (0.3, -0.2, 0.5), (0.0, 0.1, -0.1), 0.6
    cr = grid_crystal(lattice, grid)
    sig = hand_sigma(lattice, grid, [va[k] - vb[k] for k in range(3)], sb, dq_mode)
    assert 0.05 < sig < 0.45   # the window edge stays inside the gap of 1 to the other terms
    d = swept_delta3(cr, [0.0, sig, -1.5 * sig], sb, dq_mode, va, vb, which)
    assert d[0] == pytest.approx(1.0 / (np.sqrt(np.pi) * sig), rel=1e-12)
    assert d[1] / d[0] == pytest.approx(np.exp(-1.0), rel=1e-9)
    assert d[2] / d[0] == pytest.approx(np.exp(-2.25), rel=1e-9)
    edge = swept_delta3(cr, [2.0 * sig * (1 - 1e-7), 2.0 * sig * (1 + 1e-7)], sb, dq_mode, va, vb, which)
    assert edge[0] > 0 and edge[1] == 0.0
    n = 800
    h = 4.4 * sig / n
    s = -2.2 * sig + h * (np.arange(n) + 0.5)
    mass = float(np.sum(swept_delta3(cr, s, sb, dq_mode, va, vb, which)) * h)
    assert mass == pytest.approx(float(__import__("math").erf(2.0)), abs=2e-4)
