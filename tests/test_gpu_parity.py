"""GPU rates vs the FP64 oracle, through the C-ABI (fp_set_modes / fp_rates4).

Modes are injected from the oracle so that both sides see identical frequencies,
eigenvectors and velocities; window decisions must then agree exactly (accepted
counts are compared as integers) and the FP64 rates to 1e-10 relative.
"""
import numpy as np
import pytest

import oracle
from paper_2104_04895_gb300 import synth
from paper_2104_04895_gb300.binding import FP_PREC_FP64, FP_PREC_MIXED

from conftest import oracle_modes

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-10
# mixed path: FP32 vertex assembly/contraction and Gaussian, exact decisions, FP64 sums.  Measured worst cases
# against the FP64 oracle: 2.7e-7 on the small grids here, 9.9e-8 (BAs 12^3), 1.8e-7 (LiCoO2 10x10x6, against the
# FP64 path), 2.2e-7 (diamond 16^3, 8 temperatures); the bound is about 10x the worst
RTOL_MIXED = 3e-6


@pytest.fixture(scope="module")
def lib():
    from paper_2104_04895_gb300 import binding
    binding.load()
    return binding


def run_gpu(binding, cr, w, e, v, temps=None, **opts):
    with binding.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        return ctx.rates4(temps if temps is not None else cr.temps, cr.scalebroad, **opts)


def compare(gpu, ref, rtol):
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    assert gpu.shape == ref.shape
    zero = ref == 0.0
    assert np.all(gpu[zero] == 0.0)
    rel = np.abs(gpu[~zero] - ref[~zero]) / np.abs(ref[~zero])
    assert rel.max(initial=0.0) <= rtol, f"max rel err {rel.max():.3e}"
    return rel.max(initial=0.0)


CASES = [
    ("sc-1x1x1", lambda: synth.simple_cubic((1, 1, 1))),
    ("diamond-1x1x1", lambda: synth.diamond_si((1, 1, 1))),
    ("sc-2x2x2", lambda: synth.simple_cubic((2, 2, 2))),
    ("sc-3x2x1", lambda: synth.simple_cubic((3, 2, 1))),
    ("diamond-3x3x2", lambda: synth.diamond_si((3, 3, 2))),
    ("bas-3x3x3", lambda: synth.zincblende_bas((3, 3, 3))),
    ("licoo2-2x2x1", lambda: synth.licoo2((2, 2, 1))),
]


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
def test_fp64_parity_small(lib, name, maker):
    cr = maker()
    w, e, v = oracle_modes(cr)
    ref, acc = oracle.rates4(cr, w, e, v)
    out, st = run_gpu(lib, cr, w, e, v)
    compare(out.reshape(len(cr.temps), -1), ref, RTOL_FP64)
    assert np.array_equal(np.array(st["accepted"]), acc)


def test_fp64_parity_workload1_full_grid(lib):
    cr = synth.workload(1)
    w, e, v = oracle_modes(cr)
    ref, acc = oracle.rates4(cr, w, e, v)
    out, st = run_gpu(lib, cr, w, e, v)
    compare(out.reshape(1, -1), ref, RTOL_FP64)
    assert np.array_equal(np.array(st["accepted"]), acc)
    assert st["candidates"] == 3 * cr.nq ** 3 * cr.nb ** 4


@pytest.mark.parametrize("tiles", [dict(block_j0=1, k1_tile=3, threads=64), dict(block_j0=3, k1_tile=7, threads=96),
                                   dict(block_j0=3, k1_tile=64, threads=128)])
def test_fp64_tilings_agree(lib, tiles):
    cr = synth.simple_cubic((4, 3, 3))
    w, e, v = oracle_modes(cr)
    ref, acc = oracle.rates4(cr, w, e, v)
    out, st = run_gpu(lib, cr, w, e, v, **tiles)
    compare(out.reshape(1, -1), ref, RTOL_FP64)
    assert np.array_equal(np.array(st["accepted"]), acc)


def test_temperature_batch_and_dq_mode(lib):
    cr = synth.licoo2((2, 2, 2))
    w, e, v = oracle_modes(cr)
    temps = [300.0, 500.0, 700.0]
    for dq_mode in (0, 1):
        ref, acc = oracle.rates4(cr, w, e, v, temps=temps, dq_mode=dq_mode)
        out, st = run_gpu(lib, cr, w, e, v, temps=temps, dq_mode=dq_mode)
        compare(out.reshape(3, -1), ref, RTOL_FP64)
        assert np.array_equal(np.array(st["accepted"]), acc)


def test_q_range_and_mask(lib):
    cr = synth.diamond_si((3, 3, 2))
    w, e, v = oracle_modes(cr)
    nb = cr.nb
    rng = np.random.Generator(np.random.PCG64(7))
    mask = (rng.random(cr.nq * nb) < 0.3).astype(np.uint8)
    sel = np.nonzero(mask)[0]
    ref, _ = oracle.rates4(cr, w, e, v, sel=sel)
    out, _ = run_gpu(lib, cr, w, e, v, mode_mask=mask)
    flat = out.reshape(-1)
    compare(flat[sel][None, :], ref, RTOL_FP64)
    assert np.all(flat[mask == 0] == 0.0)
    # q range [5, 11)
    sel = np.arange(5 * nb, 11 * nb)
    ref, _ = oracle.rates4(cr, w, e, v, sel=sel)
    out, _ = run_gpu(lib, cr, w, e, v, q_begin=5, q_end=11)
    flat = out.reshape(-1)
    compare(flat[sel][None, :], ref, RTOL_FP64)
    assert np.all(flat[:5 * nb] == 0.0) and np.all(flat[11 * nb:] == 0.0)


def test_mixed_precision_bound(lib):
    for cr in (synth.simple_cubic((4, 4, 4)), synth.diamond_si((3, 3, 3)), synth.licoo2((2, 2, 1))):
        w, e, v = oracle_modes(cr)
        ref, acc = oracle.rates4(cr, w, e, v)
        out, st = run_gpu(lib, cr, w, e, v, precision=FP_PREC_MIXED)
        err = compare(out.reshape(len(cr.temps), -1), ref, RTOL_MIXED)
        assert np.array_equal(np.array(st["accepted"]), acc)
        print(f"{cr.name} {cr.grid}: mixed max rel err {err:.3e}")


def test_quadratic_scaling_bitwise(lib):
    cr = synth.diamond_si((2, 2, 2))
    w, e, v = oracle_modes(cr)
    a, _ = run_gpu(lib, cr, w, e, v)
    b, _ = run_gpu(lib, cr.scaled_fc4(2.0), w, e, v)
    assert np.array_equal(b, 4.0 * a)
    z, _ = run_gpu(lib, cr.scaled_fc4(0.0), w, e, v)
    assert np.all(z == 0.0)


def test_workload2_full_size_sampled_modes(lib):
    """Diamond 8x8x8 (nb = 6), the benchmark's launch configuration, checked on sampled modes."""
    cr = synth.workload(2)
    w, e, v = oracle_modes(cr)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        out, st = ctx.rates4(cr.temps, cr.scalebroad)
    rng = np.random.Generator(np.random.PCG64(2104))
    sel = np.sort(rng.choice(np.arange(cr.nb, cr.nq * cr.nb), size=3, replace=False))
    ref, _ = oracle.rates4(cr, w, e, v, sel=sel)
    compare(out.reshape(1, -1)[:, sel], ref, RTOL_FP64)


def test_autotuned_tiles_and_graph_replay(lib):
    """fp_autotune picks admissible tiles; tuned and graph-replayed calls keep FP64 parity."""
    cr = synth.diamond_si((4, 4, 3))
    w, e, v = oracle_modes(cr)
    ref, acc = oracle.rates4(cr, w, e, v)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        tiles, best = ctx.autotune(cr.temps, cr.scalebroad, precision=FP_PREC_FP64)
        assert cr.nb % tiles["block_j0"] == 0 and tiles["threads"] >= tiles["block_j0"] * cr.nb ** 2 and best > 0
        outs = []
        for _ in range(3):  # first call captures the graph, the others replay it
            out, st = ctx.rates4(cr.temps, cr.scalebroad)
            assert st["tile"][0] == tiles["block_j0"]
            outs.append(out)
        plain, _ = ctx.rates4(cr.temps, cr.scalebroad, no_graph=1)
    for out in outs + [plain]:
        compare(out.reshape(1, -1), ref, RTOL_FP64)
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[0], plain)


def test_channels_match_the_oracle_per_process(lib):
    """fp_rates4_channels: the ++, +- and -- parts of Eq. 4phgamma against the oracle, and their sum
    against fp_rates4; fp_rates4 with a one-class process_mask gives the same channel."""
    cr = synth.simple_cubic((3, 3, 3))
    w, e, v = oracle_modes(cr)
    temps = [300.0, 700.0]
    nT = len(temps)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        ch, st = ctx.rates4_channels(temps, cr.scalebroad)
        tot, st_tot = ctx.rates4(temps, cr.scalebroad)
        one, st_one = ctx.rates4(temps, cr.scalebroad, process_mask=2, no_graph=1)
        chm, _ = ctx.rates4_channels(temps, cr.scalebroad, precision=FP_PREC_MIXED)
        for bad in (-1, 8):
            with pytest.raises(lib.FourPhononError):
                ctx.rates4(temps, cr.scalebroad, process_mask=bad)
        with pytest.raises(lib.FourPhononError):
            ctx.rates4_channels(temps, cr.scalebroad, process_mask=1)
    assert ch.shape == (nT, 3, cr.nq, cr.nb)
    for p in range(3):
        ref, acc = oracle.rates4(cr, w, e, v, temps=temps, processes=(p,))
        assert acc[p] > 0
        compare(ch[:, p].reshape(nT, -1), ref, RTOL_FP64)
        compare(chm[:, p].reshape(nT, -1), ref, RTOL_MIXED)
        assert st["accepted"][p] == acc[p]
    assert st["accepted"] == st_tot["accepted"]
    np.testing.assert_allclose(ch.sum(axis=1), tot, rtol=1e-12, atol=0.0)
    assert np.array_equal(one, ch[:, 1])
    assert st_one["accepted"][0] == 0 and st_one["accepted"][2] == 0
    assert st_one["candidates"] == st_tot["candidates"] / 3


@pytest.mark.parametrize("window,sigma_min", [(3.5, 1e-10), (2.0, 0.2), (0.5, 1e-10)])
def test_window_and_sigma_min_options(lib, window, sigma_min):
    """Window and sigma_min away from their defaults: a window above 2 sends Gaussian arguments past the FP64
    exp table (u > 4), a large sigma_min makes many terms take delta := 1, a narrow window accepts few."""
    cr = synth.diamond_si((3, 3, 2))
    w, e, v = oracle_modes(cr)
    ref, acc = oracle.rates4(cr, w, e, v, window=window, sigma_min=sigma_min)
    for prec, rtol in ((FP_PREC_FP64, RTOL_FP64), (FP_PREC_MIXED, RTOL_MIXED)):
        out, st = run_gpu(lib, cr, w, e, v, precision=prec, window=window, sigma_min=sigma_min)
        compare(out.reshape(1, -1), ref, rtol)
        assert np.array_equal(np.array(st["accepted"]), acc)


def degenerate_mean(rates, omega):
    """rates (nT, N, nb) averaged over each q's degenerate branch sets (|dw| <= 1e-8 max w, chained)."""
    out = np.array(rates, dtype=np.float64, copy=True)
    tol = 1e-8 * np.max(omega)
    nb = omega.shape[1]
    for q in range(omega.shape[0]):
        j = 0
        while j < nb:
            k = j
            while k + 1 < nb and omega[q, k + 1] - omega[q, k] <= tol:
                k += 1
            out[:, q, j:k + 1] = rates[:, q, j:k + 1].mean(axis=1, keepdims=True)
            j = k + 1
    return out


@pytest.mark.parametrize("maker", [lambda: synth.simple_cubic((4, 4, 4), symmetric=True),
                                   lambda: synth.diamond_si((4, 4, 4), symmetric=True)],
                         ids=["sc-sym-4x4x4", "diamond-sym-4x4x4"])
def test_irreducible_wedge_matches_the_full_grid(lib, maker):
    """fp_rates4_irreducible on point-group symmetric force constants: one q per star, mapped to the grid,
    equals the full-grid rates averaged over degenerate sets."""
    cr = maker()
    w, e, v = oracle_modes(cr)
    ops = synth.point_group_ops(cr)
    temps = [300.0, 600.0]
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        full, st_full = ctx.rates4(temps, cr.scalebroad)
        irr, st_irr, nirr = ctx.rates4_irreducible(ops, temps, cr.scalebroad)
        irr_m, _, _ = ctx.rates4_irreducible(ops, temps, cr.scalebroad, precision=FP_PREC_MIXED)
        with pytest.raises(lib.FourPhononError):
            ctx.rates4_irreducible(ops, temps, cr.scalebroad, dq_mode=1)
        with pytest.raises(lib.FourPhononError):
            ctx.rates4_irreducible(ops, temps, cr.scalebroad, q_end=3)
    assert nirr == lib.star_table(cr.grid, ops)[1] and nirr < cr.nq
    ref = degenerate_mean(full, np.asarray(w).reshape(cr.nq, cr.nb))
    compare(irr.reshape(len(temps), -1), ref.reshape(len(temps), -1), 1e-9)
    compare(irr_m.reshape(len(temps), -1), ref.reshape(len(temps), -1), RTOL_MIXED)
    assert st_irr["candidates"] == st_full["candidates"] * nirr / cr.nq


@pytest.mark.parametrize("maker", [lambda: synth.simple_cubic((4, 4, 4)), lambda: synth.diamond_si((3, 3, 2)),
                                   lambda: synth.licoo2((2, 2, 2))], ids=["sc-4x4x4", "diamond-3x3x2", "licoo2-2x2x2"])
def test_normal_and_umklapp_match_the_oracle(lib, maker):
    """fp_rates4_nu: normal and Umklapp parts against the oracle's split (same reading of Q, implemented
    separately on each side), counts as integers; nu_select on fp_rates4 gives the same parts."""
    cr = maker()
    w, e, v = oracle_modes(cr)
    temps = [300.0, 700.0]
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        nu, st = ctx.rates4_nu(temps, cr.scalebroad)
        nu_m, _ = ctx.rates4_nu(temps, cr.scalebroad, precision=FP_PREC_MIXED)
        umk, st_u = ctx.rates4(temps, cr.scalebroad, nu_select=2, no_graph=1)
        with pytest.raises(lib.FourPhononError):
            ctx.rates4(temps, cr.scalebroad, nu_select=3)
        with pytest.raises(lib.FourPhononError):
            ctx.rates4_nu(temps, cr.scalebroad, nu_select=1)
    assert nu.shape == (len(temps), 2, cr.nq, cr.nb)
    total = np.zeros(3)
    for k, part in enumerate(("normal", "umklapp")):
        ref, acc = oracle.rates4(cr, w, e, v, temps=temps, nu=part)
        compare(nu[:, k].reshape(len(temps), -1), ref, RTOL_FP64)
        compare(nu_m[:, k].reshape(len(temps), -1), ref, RTOL_MIXED)
        total += acc
    assert np.array_equal(np.array(st["accepted"]), total)
    assert np.array_equal(umk, nu[:, 1])


def _neg_index(grid, q):
    g = np.unravel_index(q, grid)
    return int(np.ravel_multi_index(tuple((-np.asarray(g)) % np.asarray(grid)), grid))


@pytest.mark.parametrize("maker", [lambda: synth.diamond_si((3, 3, 2)), lambda: synth.zincblende_bas((4, 3, 3)),
                                   lambda: synth.licoo2((2, 2, 2)), lambda: synth.simple_cubic((4, 4, 4))],
                         ids=["diamond-3x3x2", "bas-4x3x3", "licoo2-2x2x2", "sc-4x4x4"])
def test_time_reversal_evaluates_half_the_grid(lib, maker):
    """The default path evaluates one point of each pair {q, -q} (e^{-lambda} = conj e^{lambda}, Sec. 2.2) and
    writes its rates at both; every q evaluated separately (no_time_reversal = 1) and the oracle agree with it,
    accepted counts are exact integers, and the screened candidates drop to (N + self-conjugate points) / 2N."""
    cr = maker()
    w, e, v = oracle_modes(cr)
    temps = [300.0, 800.0]
    ref, acc = oracle.rates4(cr, w, e, v, temps=temps)
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        fold, st_f = ctx.rates4(temps, cr.scalebroad)
        every, st_e = ctx.rates4(temps, cr.scalebroad, no_time_reversal=1)
        fold_m, st_fm = ctx.rates4(temps, cr.scalebroad, precision=FP_PREC_MIXED)
        with pytest.raises(lib.FourPhononError):
            ctx.rates4(temps, cr.scalebroad, no_time_reversal=2)
    nT = len(temps)
    compare(fold.reshape(nT, -1), ref, RTOL_FP64)
    compare(every.reshape(nT, -1), ref, RTOL_FP64)
    compare(fold_m.reshape(nT, -1), ref, RTOL_MIXED)
    for st in (st_f, st_e, st_fm):
        assert np.array_equal(np.array(st["accepted"]), acc)
        assert st["candidates"] == 3 * cr.nq ** 3 * cr.nb ** 4
    N = cr.nq
    selfconj = sum(1 for q in range(N) if _neg_index(cr.grid, q) == q)
    assert st_e["candidates_executed"] == st_e["candidates"]
    assert st_f["candidates_executed"] == st_f["candidates"] * (N + selfconj) / (2 * N)
    if selfconj < N:  # on a grid of 2s every point is its own -q and nothing folds
        assert st_f["vertex_entries"] < st_e["vertex_entries"] and st_f["flops"] < st_e["flops"]
        assert st_f["terms_executed"] < st_e["terms_executed"]
    else:
        assert st_f["vertex_entries"] == st_e["vertex_entries"]
    for q in range(N):
        assert np.array_equal(fold[:, q], fold[:, _neg_index(cr.grid, q)])


@pytest.mark.parametrize("maker,tiles", [(lambda: synth.diamond_si((3, 3, 2)), {}),
                                         (lambda: synth.zincblende_bas((3, 3, 3)), {}),
                                         (lambda: synth.diamond_si((4, 4, 3)), dict(block_j0=3, k1_tile=2, threads=128)),
                                         (lambda: synth.diamond_si((3, 2, 2)), dict(block_j0=1, k1_tile=1, threads=64))],
                         ids=["diamond-3x3x2", "bas-3x3x3", "diamond-4x4x3-J3", "diamond-3x2x2-J1"])
def test_tensor_core_contraction(lib, maker, tiles):
    """The mixed path with the per-q'' contraction T = A conj(E3) on the tensor cores (tcgen05 kind::tf32, 3xTF32,
    FP32 accumulation in tensor memory): within the mixed bound of the oracle, exact accepted counts, one and
    three temperatures, and row tiles that fill two, one or a fraction of an M = 128 tile."""
    cr = maker()
    w, e, v = oracle_modes(cr)
    for temps in ([300.0], [300.0, 600.0, 900.0]):
        ref, acc = oracle.rates4(cr, w, e, v, temps=temps)
        out, st = run_gpu(lib, cr, w, e, v, temps=temps, precision=FP_PREC_MIXED, tensor_cores=1, **tiles)
        simt, _ = run_gpu(lib, cr, w, e, v, temps=temps, precision=FP_PREC_MIXED, **tiles)
        err = compare(out.reshape(len(temps), -1), ref, RTOL_MIXED)
        assert np.array_equal(np.array(st["accepted"]), acc)
        print(f"{cr.name} {cr.grid} nT={len(temps)}: tensor-core mixed err {err:.2e}, "
              f"CUDA-core mixed err {compare(simt.reshape(len(temps), -1), ref, RTOL_MIXED):.2e}")


def test_tensor_cores_reject_other_paths(lib):
    cr = synth.simple_cubic((2, 2, 2))
    w, e, v = oracle_modes(cr)
    with pytest.raises(lib.FourPhononError):
        run_gpu(lib, cr, w, e, v, precision=FP_PREC_MIXED, tensor_cores=1)   # nb = 3
    cr = synth.diamond_si((2, 2, 2))
    w, e, v = oracle_modes(cr)
    with pytest.raises(lib.FourPhononError):
        run_gpu(lib, cr, w, e, v, precision=FP_PREC_FP64, tensor_cores=1)
    with pytest.raises(lib.FourPhononError):
        run_gpu(lib, cr, w, e, v, precision=FP_PREC_MIXED, tensor_cores=2)


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
def test_double_float_parity_small(lib, name, maker):
    """FP_PREC_DOUBLE_FLOAT (the FP64 path with its vertex contraction in pairs of floats on the FP32 pipes) holds
    the FP64 bar: 1e-10 of the oracle and exact accepted counts."""
    from paper_2104_04895_gb300.binding import FP_PREC_DOUBLE_FLOAT
    cr = maker()
    w, e, v = oracle_modes(cr)
    ref, acc = oracle.rates4(cr, w, e, v)
    out, st = run_gpu(lib, cr, w, e, v, precision=FP_PREC_DOUBLE_FLOAT)
    err = compare(out.reshape(len(cr.temps), -1), ref, RTOL_FP64)
    assert np.array_equal(np.array(st["accepted"]), acc)
    print(f"{name}: double-float max rel err {err:.2e}")


@pytest.mark.parametrize("tiles", [dict(block_j0=1, k1_tile=3, threads=64), dict(block_j0=3, k1_tile=7, threads=96)])
def test_double_float_tilings_temperatures_and_dq_mode(lib, tiles):
    from paper_2104_04895_gb300.binding import FP_PREC_DOUBLE_FLOAT
    cr = synth.licoo2((2, 2, 2))
    w, e, v = oracle_modes(cr)
    temps = [300.0, 500.0, 700.0]
    for dq_mode in (0, 1):
        ref, acc = oracle.rates4(cr, w, e, v, temps=temps, dq_mode=dq_mode)
        out, st = run_gpu(lib, cr, w, e, v, temps=temps, dq_mode=dq_mode, precision=FP_PREC_DOUBLE_FLOAT)
        compare(out.reshape(3, -1), ref, RTOL_FP64)
        assert np.array_equal(np.array(st["accepted"]), acc)
    cr = synth.simple_cubic((4, 3, 3))
    w, e, v = oracle_modes(cr)
    ref, acc = oracle.rates4(cr, w, e, v)
    out, st = run_gpu(lib, cr, w, e, v, precision=FP_PREC_DOUBLE_FLOAT, **tiles)
    compare(out.reshape(1, -1), ref, RTOL_FP64)
    assert np.array_equal(np.array(st["accepted"]), acc)


GENERAL_CASES = [
    ("sc-3x3x2-general", lambda: synth.simple_cubic((3, 3, 2), general=True)),
    ("diamond-3x3x2-general", lambda: synth.diamond_si((3, 3, 2), general=True)),
    ("bas-3x2x2-general", lambda: synth.zincblende_bas((3, 2, 2), general=True)),
    ("licoo2-2x2x1-general", lambda: synth.licoo2((2, 2, 1), general=True)),
]


@pytest.mark.parametrize("name,maker", GENERAL_CASES, ids=[c[0] for c in GENERAL_CASES])
def test_general_phi4_in_every_precision(lib, name, maker):
    """Phi4 that is not symmetric in the Cartesian indices of one quartet (the general per-bond form, which keeps
    Eq. TS): the order in which the library's assembly pairs the Cartesian indices with the four legs of Eq. V4 is
    checked against the oracle's.  FP64 and double-float at 1e-10, mixed (and, for six branches, its tensor-core
    contraction) within the mixed bound; accepted counts exact in all."""
    from paper_2104_04895_gb300.binding import FP_PREC_DOUBLE_FLOAT
    cr = maker()
    w, e, v = oracle_modes(cr)
    temps = [300.0, 700.0]
    ref, acc = oracle.rates4(cr, w, e, v, temps=temps)
    runs = [("fp64", dict(precision=FP_PREC_FP64), RTOL_FP64),
            ("double-float", dict(precision=FP_PREC_DOUBLE_FLOAT), RTOL_FP64),
            ("mixed", dict(precision=FP_PREC_MIXED), RTOL_MIXED)]
    if cr.nb == 6:
        runs.append(("mixed, tensor cores", dict(precision=FP_PREC_MIXED, tensor_cores=1), RTOL_MIXED))
    for label, opts, rtol in runs:
        out, st = run_gpu(lib, cr, w, e, v, temps=temps, **opts)
        err = compare(out.reshape(len(temps), -1), ref, rtol)
        assert np.array_equal(np.array(st["accepted"]), acc), label
        print(f"{name} {label}: max rel err {err:.2e}")


def test_empty_selections_and_temperature_limits(lib):
    """Edge cases of the selection and the temperature batch: an all-zero mode mask and an empty q range write zeros
    over the whole output (a NaN-filled device buffer) and count no candidates; eight temperatures (the batch
    limit) match the oracle; nine are rejected, and the context stays usable."""
    import torch
    cr = synth.diamond_si((3, 2, 2))
    w, e, v = oracle_modes(cr)
    N, nb = cr.nq, cr.nb
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        out = torch.full((N * nb,), float("nan"), dtype=torch.float64, device="cuda")
        for opts in (dict(mode_mask=np.zeros(N * nb, np.uint8)), dict(q_begin=4, q_end=4)):
            for prec in (FP_PREC_FP64, FP_PREC_MIXED):
                out.fill_(float("nan"))
                st = ctx.rates4_device([300.0], out.data_ptr(), cr.scalebroad, precision=prec, **opts)
                torch.cuda.synchronize()
                assert torch.all(out == 0.0).item(), (opts.keys(), prec)
                assert st["candidates"] == 0 and sum(st["accepted"]) == 0
        temps = list(np.linspace(300.0, 1000.0, 8))
        ref, acc = oracle.rates4(cr, w, e, v, temps=temps)
        got, st = ctx.rates4(temps, cr.scalebroad)
        compare(got.reshape(8, -1), ref, RTOL_FP64)
        assert np.array_equal(np.array(st["accepted"]), acc)
        with pytest.raises(lib.FourPhononError) as ei:
            ctx.rates4(list(np.linspace(300.0, 1000.0, 9)), cr.scalebroad)
        assert ei.value.code == lib.FP_EINVAL
        again, _ = ctx.rates4(temps, cr.scalebroad)
        assert np.array_equal(again, got)
