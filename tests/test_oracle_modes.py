"""Pins of the oracle's harmonic step (frequencies, eigenvectors, velocities).

Pinned against things other than the oracle itself: the textbook closed form of the
simple-cubic dynamical matrix with central nearest- and next-nearest-neighbour
springs, finite differences of those closed-form frequencies, the eigen-equation of
an independently assembled real-space matrix, and exact time-reversal relations.
"""
import numpy as np
import pytest

import oracle.modes as om
from paper_2104_04895_gb300 import synth
from conftest import oracle_modes


# SI values (CODATA 2018, exact where defined), independent of the oracle's own conversion constant: a dynamical
# matrix in eV / (A^2 amu) times EV_J / (ANG_M^2 AMU_KG) is in s^-2, and 1e-24 turns s^-2 into ps^-2
EV_J = 1.602176634e-19
AMU_KG = 1.66053906660e-27
ANG_M = 1e-10
TO_PS2 = EV_J / (ANG_M ** 2 * AMU_KG) * 1e-24


def sc_closed_form(qc, a=3.0, k1=1.0, k2=0.5, M=28.0855):
    """Textbook SC dynamical matrix: D_xx = 2/M [k1 (1 - cx) + k2 (2 - cx cy - cx cz)], D_xy = 2 k2 sx sy / M."""
    c = np.cos(qc * a)
    s = np.sin(qc * a)
    D = np.zeros((3, 3))
    for x in range(3):
        y, z = (x + 1) % 3, (x + 2) % 3
        D[x, x] = 2.0 / M * (k1 * (1 - c[x]) + k2 * (2 - c[x] * c[y] - c[x] * c[z]))
        D[x, y] = D[y, x] = 2.0 * k2 / M * s[x] * s[y]
    return D


def test_sc_frequencies_match_closed_form():
    cr = synth.simple_cubic((4, 4, 4))
    w, e, v = oracle_modes(cr)
    B = om.reciprocal(cr.lattice)
    G = om.grid_points(cr.grid)
    for q in range(cr.nq):
        qc = (G[q] / np.array(cr.grid)) @ B
        ev = np.sort(np.linalg.eigvalsh(sc_closed_form(qc)))
        ref = np.sqrt(np.clip(ev * TO_PS2, 0, None))
        if q == 0:
            ref[:3] = 0.0
        np.testing.assert_allclose(w[q], ref, rtol=1e-12, atol=1e-9)


def test_sc_velocities_match_finite_differences():
    cr = synth.simple_cubic((5, 5, 5))
    w, e, v = oracle_modes(cr)
    B = om.reciprocal(cr.lattice)
    G = om.grid_points(cr.grid)
    h = 1e-6
    checked = 0
    for q in range(1, cr.nq):
        qc = (G[q] / np.array(cr.grid)) @ B
        ws = np.sqrt(np.sort(np.linalg.eigvalsh(sc_closed_form(qc))) * TO_PS2)
        if np.min(np.diff(ws)) < 1e-3 * ws.max():
            continue  # finite differences are not defined on degenerate sets
        if np.all(np.abs(v[q]) == 0):
            continue
        fd = np.zeros((3, 3))
        for c in range(3):
            dq = np.zeros(3)
            dq[c] = h
            wp = np.sqrt(np.sort(np.linalg.eigvalsh(sc_closed_form(qc + dq))) * TO_PS2)
            wm = np.sqrt(np.sort(np.linalg.eigvalsh(sc_closed_form(qc - dq))) * TO_PS2)
            fd[:, c] = (wp - wm) / (2 * h)
        np.testing.assert_allclose(v[q], fd, rtol=1e-6, atol=1e-6)
        checked += 1
    assert checked > 10


@pytest.mark.parametrize("maker", [lambda: synth.diamond_si((4, 4, 4)), lambda: synth.licoo2((3, 3, 2)),
                                   lambda: synth.zincblende_bas((3, 3, 3))])
def test_eigen_equation_and_orthonormality(maker):
    cr = maker()
    w, e, v = oracle_modes(cr)
    G = om.grid_points(cr.grid)
    nb = cr.nb
    for q in range(cr.nq):
        # independent real-space assembly: sum over pair blocks with a direct loop
        D = np.zeros((nb, nb), complex)
        for idx, val in zip(cr.fc2_idx, cr.fc2_val):
            i, j = idx[0], idx[1]
            ang = 2 * np.pi * sum(G[q][a] * idx[2 + a] / cr.grid[a] for a in range(3))
            for al in range(3):
                for be in range(3):
                    D[3 * i + al, 3 * j + be] += val[3 * al + be] * complex(np.cos(ang), np.sin(ang)) / np.sqrt(
                        cr.mass[i] * cr.mass[j])
        for b in range(nb):
            lhs = D @ e[q, b]
            rhs = (w[q, b] ** 2 / TO_PS2) * e[q, b]
            assert np.abs(lhs - rhs).max() < 1e-10 * max(1.0, np.abs(D).max())
        np.testing.assert_allclose(e[q] @ e[q].conj().T, np.eye(nb), atol=1e-12)


def test_time_reversal_is_exact():
    cr = synth.diamond_si((4, 4, 4))
    w, e, v = oracle_modes(cr)
    G = om.grid_points(cr.grid)
    ng = np.array(cr.grid)
    for q in range(cr.nq):
        g = (-G[q]) % ng
        p = (g[0] * ng[1] + g[1]) * ng[2] + g[2]
        assert np.array_equal(w[p], w[q])
        assert np.array_equal(e[p], e[q].conj())
        assert np.array_equal(v[p], -v[q])
        if p == q:
            assert np.all(e[q].imag == 0) and np.all(v[q] == 0)


def test_gamma_acoustic_zero_and_stable():
    for k in (1, 2, 3, 4):
        cr = synth.workload(k).with_grid((2, 2, 2))
        w, e, v = oracle_modes(cr)
        assert np.all(w[0, :3] == 0.0)
        assert np.all(w[0, 3:] > 0.0)
        assert np.all(w[1:] > 0.0)


@pytest.mark.parametrize("maker", [lambda: synth.zincblende_bas((2, 2, 2)), lambda: synth.diamond_si((2, 2, 2))])
def test_gamma_optical_frequency_is_the_reduced_mass_closed_form(maker):
    """Two atoms per cell, nearest-neighbour springs along the four tetrahedral bonds n (central k_c = 1, transverse
    k_t = 0.25 eV/A^2) and next-nearest springs within each sublattice: at Gamma the sublattice springs cancel by
    the sum rule, the bonds give the coupling block a I with a = k_c sum n n^T + k_t sum (I - n n^T) = 4/3 k_c +
    8/3 k_t, and the three optical modes have omega^2 = a (1/M_1 + 1/M_2) (the textbook diatomic result with the
    reduced mass); the acoustic ones are zero."""
    cr = maker()
    w, e, v = oracle_modes(cr)
    a = 4.0 / 3.0 * 1.0 + 8.0 / 3.0 * 0.25
    w_opt = np.sqrt(a * (1.0 / cr.mass[0] + 1.0 / cr.mass[1]) * TO_PS2)
    assert np.all(w[0, :3] == 0.0)
    np.testing.assert_allclose(w[0, 3:], w_opt, rtol=1e-12)
