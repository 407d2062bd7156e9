"""Pins of the oracle's RTA thermal conductivity (the kinetic form fed by the rates of Eq. tao0)."""
import numpy as np

import oracle
from paper_2104_04895_gb300 import synth
from conftest import oracle_modes


def test_high_temperature_limit_is_kinetic_theory():
    """x -> 0: each mode carries k_B, so kappa = k_B v^2 tau / (N V) (kinetic theory with the classical heat
    capacity); one mode with v along x, N = 2 cells of 27 A^3."""
    lattice = 3.0 * np.eye(3)
    omega = np.array([[0.0, 0.0, 10.0], [0.0, 0.0, 0.0]])
    vel = np.zeros((2, 3, 3))
    vel[0, 2] = [20.0, 0.0, 0.0]
    rates = np.full((1, 2, 3), 2.0)
    k = oracle.kappa_rta(lattice, omega, vel, [1e7], rates)
    expect = 1.380649e-23 * (20.0 * 100.0) ** 2 * (0.5e-12) / (2 * 27.0e-30)
    np.testing.assert_allclose(k[0, 0, 0], expect, rtol=1e-8)
    assert np.count_nonzero(k) == 1


def test_kappa_inverse_in_the_rates_and_isotropic_in_cubic_crystals():
    cr = synth.simple_cubic((4, 4, 4), symmetric=True)
    w, e, v = oracle_modes(cr)
    temps = [100.0, 300.0]
    rates = np.ones((2, cr.nq, cr.nb))
    k1 = oracle.kappa_rta(cr.lattice, w, v, temps, rates)
    k2 = oracle.kappa_rta(cr.lattice, w, v, temps, 2.0 * rates)
    np.testing.assert_allclose(k2, 0.5 * k1, rtol=1e-14, atol=0.0)
    for t in range(2):
        d = np.diag(k1[t])
        np.testing.assert_allclose(d, d.mean(), rtol=1e-10)
        assert np.abs(k1[t] - np.diag(d)).max() <= 1e-10 * d.mean()
    # the heat capacity falls with T: a lower T gives a smaller kappa at equal rates
    assert k1[0, 0, 0] < k1[1, 0, 0]
