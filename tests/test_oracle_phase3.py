"""Pins of the oracle's three-phonon-like phase space (surrogate features; Eq. 3phgamma's
energy and Bose structure without |V3|^2): an independent vectorised enumeration, and a
single-q closed form with injected frequencies and zero velocities."""
import numpy as np
import pytest

import oracle
import oracle.modes as om
from paper_2104_04895_gb300 import synth
from conftest import oracle_modes


def test_single_q_closed_form():
    cr = synth.diamond_si((1, 1, 1))
    omega = np.array([[3.0, 1.0, 2.0, 5.0, 4.0, 7.0]])
    vel = np.zeros((1, 6, 3))
    T = 300.0
    p3, wp3 = oracle.phase3(cr, omega, vel, temps=[T])
    n = np.array([oracle.bose(w, T) for w in omega[0]])
    for lam in range(6):
        w = omega[0, lam]
        ep = ew = 0.0
        for j1 in range(6):
            for j2 in range(6):
                w1, w2 = omega[0, j1], omega[0, j2]
                if w + w1 - w2 == 0.0:
                    ep += 1.0
                    ew += (n[j1] - n[j2]) / (w * w1 * w2)
                if w - w1 - w2 == 0.0:
                    ep += 0.5
                    ew += 0.5 * (n[j1] + n[j2] + 1.0) / (w * w1 * w2)
        assert p3[lam] == pytest.approx(ep, rel=1e-14, abs=0)
        assert wp3[0, lam] == pytest.approx(ew, rel=1e-12, abs=0)
    assert p3.max() > 0


def test_vectorised_enumeration():
    cr = synth.simple_cubic((3, 3, 4))
    w, e, v = oracle_modes(cr)
    nb, N = cr.nb, cr.nq
    G = om.grid_points(cr.grid)
    ng = np.array(cr.grid)
    B = om.reciprocal(cr.lattice)
    dq = (abs(np.linalg.det(B)) / N) ** (1.0 / 3.0)
    sel = [nb * 5 + 1, nb * 17 + 2, nb * 30]
    T = 500.0
    p3, wp3 = oracle.phase3(cr, w, v, temps=[T], sel=sel)
    nbose = 1.0 / np.expm1(6.582119569e-4 * np.where(w > 0, w, 1.0) / (8.617333262e-5 * T))
    for k, m in enumerate(sel):
        q, j = divmod(m, nb)
        ep = ew = 0.0
        for sgn in (1, -1):
            g2 = (G[q][None, :] + sgn * G) % ng
            q2 = (g2[:, 0] * ng[1] + g2[:, 1]) * ng[2] + g2[:, 2]
            W1 = w[:, :, None]
            W2 = w[q2][:, None, :]
            dw = (w[q, j] + sgn * W1) - W2
            d = v[:, :, None, :] - v[q2][:, None, :, :]
            sig = np.sqrt((d[..., 0] ** 2 + d[..., 1] ** 2) + d[..., 2] ** 2) * dq
            ok = (np.abs(dw) <= 2.0 * np.where(sig < 1e-10, 1e-10, sig)) & (W1 > 0) & (W2 > 0)
            delta = np.where(sig < 1e-10, 1.0, np.exp(-(dw / np.where(sig > 0, sig, 1)) ** 2) /
                             (np.sqrt(np.pi) * np.where(sig > 0, sig, 1)))
            n1 = nbose[:, :, None]
            n2 = nbose[q2][:, None, :]
            if sgn > 0:
                ep += np.sum(np.where(ok, delta, 0.0))
                ew += np.sum(np.where(ok, (n1 - n2) * delta / (w[q, j] * W1 * W2), 0.0))
            else:
                ep += 0.5 * np.sum(np.where(ok, delta, 0.0))
                ew += 0.5 * np.sum(np.where(ok, (n1 + n2 + 1) * delta / (w[q, j] * W1 * W2), 0.0))
        assert p3[k] == pytest.approx(ep / N, rel=1e-10)
        assert wp3[0, k] == pytest.approx(ew / N, rel=1e-10)
