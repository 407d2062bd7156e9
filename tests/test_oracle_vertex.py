"""Pins of the oracle's fourth-order vertex (Eq. V4 with the momentum rule of Eq. tao0's text).

* brute force: the Born-von Karman supercell sum over every atom quartet equals Eq. V4
  on tiny grids for the three processes, and vanishes when momentum is not conserved;
* symmetry: the vertex is symmetric under permutations of its four legs (transposition
  symmetry, Sec. 2.3, Eq. TS, plus translation invariance);
* e^{-lambda} = e at -q: V+-(q, q', q'') = V++(q, q', -q''), V--(q, q', q'') = V++(q, -q', -q'');
* linearity in Phi4.
"""
import numpy as np
import pytest

import oracle
import oracle.brute as brute
import oracle.modes as om
from paper_2104_04895_gb300 import synth
from conftest import oracle_modes

S = {0: (1, 1), 1: (1, -1), 2: (-1, -1)}


def neg(cr, q):
    G = om.grid_points(cr.grid)
    ng = np.array(cr.grid)
    g = (-G[q]) % ng
    return int((g[0] * ng[1] + g[1]) * ng[2] + g[2])


def third(cr, q, q1, q2, s1, s2):
    G = om.grid_points(cr.grid)
    ng = np.array(cr.grid)
    g = (G[q] + s1 * G[q1] + s2 * G[q2]) % ng
    return int((g[0] * ng[1] + g[1]) * ng[2] + g[2])


CASES = [
    lambda: synth.simple_cubic((1, 1, 1)),
    lambda: synth.simple_cubic((2, 2, 2)),
    lambda: synth.simple_cubic((3, 2, 1)),
    lambda: synth.diamond_si((2, 1, 1)),
    lambda: synth.diamond_si((2, 2, 1)),
    lambda: synth.zincblende_bas((2, 2, 2)),
    # the general Phi4 form: not symmetric in the Cartesian indices of one quartet, so the index order of Eq. V4
    # (alpha with atom i, beta with j, gamma with k, theta with l) is tested
    lambda: synth.diamond_si((2, 2, 1), general=True),
    lambda: synth.zincblende_bas((2, 1, 1), general=True),
]


@pytest.mark.parametrize("maker", CASES)
def test_vertex_equals_supercell_brute_force(maker, rng):
    cr = maker()
    w, e, v = oracle_modes(cr)
    P = brute.supercell_phi4(cr)
    N = cr.nq
    for trial in range(4):
        q, q1, q2 = (int(x) for x in rng.integers(0, N, size=3))
        for pr in range(3):
            s1, s2 = S[pr]
            V, q3 = oracle.v4(cr, e, q, q1, q2, pr)
            assert q3 == third(cr, q, q1, q2, s1, s2)
            Vb = brute.vertex(cr, P, e, q, q1, q2, q3, conj1=s1 < 0, conj2=s2 < 0)
            # natural magnitude of a vertex: sum |Phi4| / M^2 (all-acoustic Gamma vertices vanish by the ASR)
            natural = np.abs(cr.fc4_val).sum() / cr.mass.min() ** 2
            scale = max(np.abs(Vb).max(), 1e-3 * natural)
            assert np.abs(V - Vb).max() <= 1e-12 * scale, (q, q1, q2, pr)


def test_supercell_sum_vanishes_off_momentum_shell(rng):
    cr = synth.diamond_si((2, 2, 1))
    w, e, v = oracle_modes(cr)
    P = brute.supercell_phi4(cr)
    q, q1, q2 = 1, 2, 3
    q3 = third(cr, q, q1, q2, 1, 1)
    Vok = brute.vertex(cr, P, e, q, q1, q2, q3)
    bad = (q3 + 1) % cr.nq
    Vbad = brute.vertex(cr, P, e, q, q1, q2, bad)
    assert np.abs(Vok).max() > 1e-3
    assert np.abs(Vbad).max() < 1e-12 * np.abs(Vok).max()


@pytest.mark.parametrize("general", [False, True], ids=["bond-phi4", "general-phi4"])
def test_vertex_leg_permutations(rng, general):
    cr = synth.diamond_si((3, 3, 2), general=general)
    w, e, v = oracle_modes(cr)
    N = cr.nq
    for trial in range(3):
        q, k1, k2 = (int(x) for x in rng.integers(0, N, size=3))
        W, k3 = oracle.v4(cr, e, q, k1, k2, 0)
        scale = np.abs(W).max()
        # swap the two partner legs
        W2, k3b = oracle.v4(cr, e, q, k2, k1, 0)
        assert k3b == k3
        assert np.abs(W - W2.transpose(0, 2, 1, 3)).max() <= 1e-12 * scale
        # swap the mode leg with the first partner
        W3, k3c = oracle.v4(cr, e, k1, q, k2, 0)
        assert k3c == k3
        assert np.abs(W - W3.transpose(1, 0, 2, 3)).max() <= 1e-12 * scale
        # swap the first partner with the outgoing leg: (q; -k3, k2) has third momentum -k1
        W4, k1b = oracle.v4(cr, e, q, neg(cr, k3), k2, 0)
        assert k1b == neg(cr, k1)
        assert np.abs(W - W4.transpose(0, 3, 2, 1)).max() <= 1e-12 * scale


def test_processes_share_one_vertex(rng):
    cr = synth.zincblende_bas((3, 3, 3))
    w, e, v = oracle_modes(cr)
    N = cr.nq
    for trial in range(3):
        q, q1, q2 = (int(x) for x in rng.integers(0, N, size=3))
        Vpm, _ = oracle.v4(cr, e, q, q1, q2, 1)
        Vpp, _ = oracle.v4(cr, e, q, q1, neg(cr, q2), 0)
        assert np.abs(Vpm - Vpp).max() <= 1e-12 * np.abs(Vpp).max()
        Vmm, _ = oracle.v4(cr, e, q, q1, q2, 2)
        Vpp2, _ = oracle.v4(cr, e, q, neg(cr, q1), neg(cr, q2), 0)
        assert np.abs(Vmm - Vpp2).max() <= 1e-12 * np.abs(Vpp2).max()


def test_vertex_linear_in_phi4():
    cr = synth.simple_cubic((2, 2, 2))
    w, e, v = oracle_modes(cr)
    V1, _ = oracle.v4(cr, e, 1, 2, 3, 0)
    V2, _ = oracle.v4(cr.scaled_fc4(2.0), e, 1, 2, 3, 0)
    assert np.array_equal(V2, 2.0 * V1)
    V0, _ = oracle.v4(cr.scaled_fc4(0.0), e, 1, 2, 3, 0)
    assert np.all(V0 == 0)
