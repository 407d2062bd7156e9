"""Surrogate path on the GPU: phase-space features vs the oracle, network gradients vs the FP64
oracle backward pass, and the fitted surrogate vs exact rates (accuracy, exact fallback, and what
it saves)."""
import ctypes
import time

import numpy as np
import pytest

import oracle
import oracle.mlp as omlp
from paper_2104_04895_gb300 import synth

from conftest import oracle_modes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    """The binding; its load() declares every argument type (the tests use its structures)."""
    from paper_2104_04895_gb300 import binding
    binding.load()
    return binding


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


@pytest.mark.parametrize("maker", [lambda: synth.workload(1), lambda: synth.diamond_si((3, 3, 2)),
                                   lambda: synth.licoo2((3, 3, 2))])
def test_phase3_matches_oracle(lib, maker):
    cr = maker()
    w, e, v = oracle_modes(cr)
    temps = np.array([300.0, 700.0])
    p_ref, wp_ref = oracle.phase3(cr, w, v, temps=temps)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        p = np.zeros(cr.nq * cr.nb)
        wp = np.zeros((2, cr.nq * cr.nb))
        rc = ctx.L.fp_phase3(ctx.h, 2, _d(temps), cr.scalebroad, None, _d(p), _d(wp))
        assert rc == 0
    nz = p_ref != 0
    assert nz.any()
    assert np.all(p[~nz] == 0)
    assert np.max(np.abs(p[nz] - p_ref[nz]) / p_ref[nz]) <= 1e-10
    nz = wp_ref != 0
    assert np.all(wp[~nz] == 0)
    assert np.max(np.abs(wp[nz] - wp_ref[nz]) / np.abs(wp_ref[nz])) <= 1e-10


def test_network_gradient_matches_fp64_oracle(lib):
    F, B = 12, 96
    rng = np.random.Generator(np.random.PCG64(21))
    p = omlp.init_params(F, seed=4) + 0.02 * rng.normal(size=omlp.n_params(F))
    X = rng.normal(size=(B, F))
    y = rng.normal(size=B)
    loss_ref, g_ref = omlp.loss_and_grad(p, X, y, F)
    L = lib.load()
    assert L.fp_mlp_params_size(F) == p.size
    pf = p.astype(np.float32)
    Xf = X.astype(np.float32)
    yf = y.astype(np.float32)
    g = np.zeros(p.size, np.float32)
    loss = np.zeros(1, np.float32)
    assert L.fp_mlp_loss_grad(0, F, B, _f(Xf), _f(yf), _f(pf), _f(g), _f(loss)) == 0
    # FP32 kernels vs the FP64 oracle on FP32-rounded inputs
    loss_r, g_r = omlp.loss_and_grad(pf.astype(np.float64), Xf.astype(np.float64), yf.astype(np.float64), F)
    assert loss[0] == pytest.approx(loss_r, rel=1e-5)
    assert np.max(np.abs(g - g_r)) <= 1e-4 * np.max(np.abs(g_r))
    # and the gradient is that of the FP64 definition up to the FP32 rounding of the inputs
    assert np.max(np.abs(g - g_ref)) <= 2e-3 * np.max(np.abs(g_ref))


def test_surrogate_fit_exact_entries_fallback_rule_and_gain(lib):
    """The learned path: entries it evaluates exactly are the exact rates bit for bit; a bin keeps network
    rates only when its held-out error bound is within the tolerance; and the gain over the exact,
    temperature-batched path (share of entries not evaluated exactly, wall time) is measured and reported.

    On the benchmark crystals (random per-bond quartic constants) the rate field is rough on these grids
    (neighbouring q-points differ by ~25 %), so the network trained on 10 % of the modes misses the 5 %
    tolerance and the fallback keeps every bin exact; the test then checks that outcome is consistent."""
    cr = synth.diamond_si((8, 8, 8))
    temps = np.array([300.0, 500.0, 700.0, 900.0])
    L = lib.load()
    with lib.Context.from_crystal(cr) as ctx:
        ctx.modes(copy=False)
        t0 = time.perf_counter()
        exact, st = ctx.rates4(temps, cr.scalebroad, precision=lib.FP_PREC_MIXED)
        t_exact = time.perf_counter() - t0
        so = lib.fp_surrogate_opts()
        L.fp_surrogate_default_opts(ctypes.byref(so))
        rep = lib.fp_surrogate_report()
        t0 = time.perf_counter()
        assert L.fp_surrogate_fit(ctx.h, len(temps), _d(temps), cr.scalebroad, ctypes.byref(so),
                                  ctypes.byref(rep)) == 0
        t_sur = time.perf_counter() - t0
        rates = np.zeros_like(exact)
        used = np.zeros(exact.shape, np.uint8)
        assert L.fp_surrogate_rates(ctx.h, _d(rates), used.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))) == 0
    ex = exact.reshape(len(temps), -1)
    ra = rates.reshape(len(temps), -1)
    us = used.reshape(len(temps), -1).astype(bool)
    pos = ex[0] > 0
    # exact entries are the exact rates, bit for bit; zero-frequency modes stay zero
    assert np.array_equal(ra[us], ex[us])
    assert np.all(ra[:, ~pos] == 0)
    # the subsets: 10 % of the pairs {q, -q} trained, 5 % held out, each with all its positive-frequency branches
    # (the grid's pairs are nearly all of two points, so the mode shares are close to the pair shares)
    assert rep.n_modes == pos.sum()
    assert abs(rep.n_train / rep.n_modes - 0.10) < 0.02 and abs(rep.n_holdout / rep.n_modes - 0.05) < 0.02
    assert rep.n_train % cr.nb == 0 or rep.n_train % cr.nb == cr.nb - 3  # whole q-points (Gamma has 3 acoustic zeros)
    pred = (~us) & (ex > 0)
    share_exact = us[:, pos].mean()
    assert pred.sum() == round((1.0 - share_exact) * pos.sum() * len(temps))
    if rep.n_bins_fallback == rep.n_bins:
        assert not pred.any() and share_exact == 1.0
    else:
        rel = np.abs(ra[pred] - ex[pred]) / ex[pred]
        # bins kept on the network passed an upper confidence bound on held-out error <= 5 %
        assert np.median(rel) <= 0.10
    print(f"surrogate gain: {pred.sum()} of {pos.sum() * len(temps)} entries predicted (exact share {share_exact:.3f}); "
          f"held-out median rel err {rep.holdout_median_rel_err:.3f} p90 {rep.holdout_p90_rel_err:.3f}; "
          f"{rep.n_bins_fallback}/{rep.n_bins} bins exact; wall {t_sur:.2f} s vs exact {t_exact:.2f} s")


@pytest.mark.parametrize("maker", [lambda: synth.workload(1), lambda: synth.diamond_si((3, 3, 2))])
def test_phase4_matches_oracle_unit_vertex(lib, maker):
    """fp_phase4 with stride 1 is the rate sum with |V|^2 = 1 (the oracle's unit-vertex mode), over N^2."""
    cr = maker()
    w, e, v = oracle_modes(cr)
    temps = np.array([300.0, 600.0])
    ref, _ = oracle.rates4(cr, w, e, v, temps=temps, unit_vertex=True)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        wp4 = ctx.phase4(temps, cr.scalebroad, stride=1) * cr.nq ** 2
        wp4_s = ctx.phase4(temps, cr.scalebroad, stride=2) * cr.nq ** 2
    nz = ref != 0
    assert nz.any() and np.all(wp4[~nz] == 0)
    # FP32 Gaussian and Bose weights, exact decisions
    assert np.max(np.abs(wp4[nz] - ref[nz]) / ref[nz]) <= 2e-5
    # the strided estimate is of the same size (it samples every other q')
    assert 0.5 < np.median(wp4_s[nz] / ref[nz]) < 2.0


def test_surrogate_sweep_at_new_temperatures(lib):
    """Learned rates at new temperatures: anchors at 300, 650 and 1000 K for every mode, and 16 output temperatures
    (two batched evaluations for the exact path).  Exact entries are the exact rates bit for bit, the network's
    entries are checked against exact rates of every mode, bins it keeps hold the 5 % rule, and the network must
    replace exact evaluation for part of the entries (the gain over the method without it)."""
    cr = synth.diamond_si((6, 6, 6))
    anchors = [300.0, 650.0, 1000.0]
    temps = list(np.linspace(300.0, 1000.0, 16))
    with lib.Context.from_crystal(cr) as ctx:
        ctx.modes(copy=False)
        exact = np.concatenate([ctx.rates4(temps[i:i + 8], cr.scalebroad, precision=lib.FP_PREC_MIXED)[0]
                                for i in range(0, 16, 8)])
        rates, used, rep = ctx.surrogate_sweep(anchors, temps, cr.scalebroad)
        with pytest.raises(lib.FourPhononError):
            ctx.surrogate_sweep(anchors, [300.0] * 65, cr.scalebroad)
        with pytest.raises(lib.FourPhononError):
            ctx.surrogate_sweep([0.0], temps, cr.scalebroad)
    ex = exact.reshape(16, -1)
    ra = rates.reshape(16, -1)
    us = used.reshape(16, -1).astype(bool)
    pos = ex[0] > 0
    assert np.array_equal(ra[us], ex[us]) and np.all(ra[:, ~pos] == 0.0)
    pred = (~us) & (ex > 0)
    share_exact = us[:, pos].mean()
    # the gain: the network replaces exact evaluation for part of the (mode, T) entries (measured: 64 % of them on
    # this workload), at the 5 % rule on the entries it predicts
    assert pred.any() and share_exact < 0.9
    rel = np.abs(ra[pred] - ex[pred]) / ex[pred]
    assert np.median(rel) <= 0.05
    print(f"sweep: {pred.sum()} of {pos.sum() * 16} entries predicted (exact share {share_exact:.3f}); "
          f"predicted rel err median {np.median(rel):.4f} p90 {np.quantile(rel, 0.9):.4f} max {rel.max():.4f}; "
          f"held-out median {rep['holdout_median_rel_err']:.4f}; {rep['n_bins_fallback']}/{rep['n_bins']} bins exact")
    assert rep["n_train"] > 0 and rep["n_holdout"] > 0
