"""Parity at the full sizes of the benchmark workloads, in the launch configuration that bench.py times.

The oracle finishes one mode of zincblende BAs 12x12x12 (nb = 6) with its full vertex in about a minute on the
host cores, so the full-size comparison takes sampled modes (a mode mask on the GPU side, `sel` on the oracle
side) with the full (q', q'') partner sums of Eq. tao0:

* BAs 12^3: FP64 rates of four modes within 1e-10 of the oracle with exact accepted counts, the mixed path
  within its stated bound, and the exact accepted counts of five more modes against the oracle's window
  enumeration (the unit-vertex option, whose screening is the full one);
* LiCoO2 10x10x6 (nb = 12, three temperatures in one launch): exact per-mode accepted counts against the
  oracle on eight modes, the three-temperature launch equal to three one-temperature launches (two kernel
  instantiations), time reversal folded and not folded, and the mixed path against FP64.

Modes are chosen by rule, not by result: for each crystal, the lowest nonzero frequency (a Gamma-adjacent
acoustic mode), the highest frequency (top optical), a zone-boundary mode, and one seeded random mode per branch.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2104_04895_gb300 import synth
from paper_2104_04895_gb300.binding import FP_PREC_DOUBLE_FLOAT, FP_PREC_FP64, FP_PREC_MIXED

from conftest import oracle_modes

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-10
RTOL_MIXED = 3e-6
CORES = os.cpu_count() or 1


@pytest.fixture(scope="module")
def lib():
    from paper_2104_04895_gb300 import binding
    binding.load()
    return binding


def ruled_modes(cr, w, seed):
    """Mode indices: lowest positive frequency, highest frequency, the top branch at the zone-boundary point
    (N1/2, 0, 0), then one seeded random mode per branch (excluding those already taken)."""
    nb, N = cr.nb, cr.nq
    flat = np.asarray(w).reshape(-1)
    pos = np.nonzero(flat > 0)[0]
    picks = [int(pos[np.argmin(flat[pos])]), int(np.argmax(flat))]
    gzb = (cr.grid[0] // 2) * cr.grid[1] * cr.grid[2]
    picks.append(gzb * nb + nb - 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    for j in range(nb):
        while True:
            m = int(rng.integers(1, N)) * nb + j
            if m not in picks and flat[m] > 0:
                picks.append(m)
                break
    return picks


def gpu_single_mode_counts(ctx, cr, temps, modes, **opts):
    """Accepted counts (++, +-, --) of each mode alone: a mode mask with that one mode."""
    out = []
    for m in modes:
        mask = np.zeros(cr.nq * cr.nb, np.uint8)
        mask[m] = 1
        _, st = ctx.rates4(temps, cr.scalebroad, mode_mask=mask, no_graph=1, **opts)
        out.append(st["accepted"])
    return np.array(out)


def oracle_single_mode_counts(cr, w, e, v, temps, modes):
    out = []
    for m in modes:
        _, acc = oracle.rates4(cr, w, e, v, temps=temps[:1], sel=[m], unit_vertex=True, nthreads=CORES)
        out.append(acc)
    return np.array(out)


def rel_err(gpu, ref):
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    assert np.all(ref > 0)
    return float(np.max(np.abs(gpu - ref) / ref))


def test_bas_12_full_size(lib):
    cr = synth.workload(3)
    w, e, v = oracle_modes(cr)
    modes = ruled_modes(cr, w, seed=1203)
    full_vertex = modes[:4]          # lowest and highest frequency, the zone-boundary top branch, a seeded mode
    count_only = modes[4:]
    ref, acc = oracle.rates4(cr, w, e, v, sel=full_vertex, nthreads=CORES)
    mask = np.zeros(cr.nq * cr.nb, np.uint8)
    mask[full_vertex] = 1
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        out, st = ctx.rates4(cr.temps, cr.scalebroad, mode_mask=mask)
        outm, stm = ctx.rates4(cr.temps, cr.scalebroad, mode_mask=mask, precision=FP_PREC_MIXED)
        outd, std_ = ctx.rates4(cr.temps, cr.scalebroad, mode_mask=mask, precision=FP_PREC_DOUBLE_FLOAT)
        counts = gpu_single_mode_counts(ctx, cr, cr.temps, count_only)
    got = out.reshape(1, -1)[:, full_vertex]
    gotm = outm.reshape(1, -1)[:, full_vertex]
    err = rel_err(got, ref)
    errm = rel_err(gotm, ref)
    errd = rel_err(outd.reshape(1, -1)[:, full_vertex], ref)
    print(f"BAs 12^3 full size: FP64 {err:.2e}, double-float {errd:.2e}, mixed {errm:.2e} on modes {full_vertex}")
    assert err <= RTOL_FP64 and errd <= RTOL_FP64
    assert np.array_equal(np.array(std_["accepted"]), acc)
    assert errm <= RTOL_MIXED
    assert np.array_equal(np.array(st["accepted"]), acc) and np.array_equal(np.array(stm["accepted"]), acc)
    assert np.all(out.reshape(-1)[mask == 0] == 0.0)
    ref_counts = oracle_single_mode_counts(cr, w, e, v, list(cr.temps), count_only)
    assert np.array_equal(counts, ref_counts)
    print("BAs 12^3 accepted counts per mode:", ref_counts.sum(axis=1).astype(np.int64).tolist())


def test_licoo2_10x10x6_full_size_three_temperatures(lib):
    cr = synth.workload(4)
    w, e, v = oracle_modes(cr)
    temps = list(cr.temps)
    assert len(temps) == 3
    modes = ruled_modes(cr, w, seed=1004)[:8]
    mask = np.zeros(cr.nq * cr.nb, np.uint8)
    mask[modes] = 1
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        three, st3 = ctx.rates4(temps, cr.scalebroad, mode_mask=mask)
        every, ste = ctx.rates4(temps, cr.scalebroad, mode_mask=mask, no_time_reversal=1)
        ones = [ctx.rates4([T], cr.scalebroad, mode_mask=mask)[0] for T in temps]
        mixed, stm = ctx.rates4(temps, cr.scalebroad, mode_mask=mask, precision=FP_PREC_MIXED)
        counts = gpu_single_mode_counts(ctx, cr, temps, modes)
    ref_counts = oracle_single_mode_counts(cr, w, e, v, temps, modes)
    assert np.array_equal(counts, ref_counts)
    assert np.array_equal(np.array(st3["accepted"]), ref_counts.sum(axis=0))
    assert st3["accepted"] == ste["accepted"] == stm["accepted"]
    a = three.reshape(3, -1)[:, modes]
    assert np.all(a > 0)
    for t in range(3):
        np.testing.assert_allclose(ones[t].reshape(1, -1)[0, modes], a[t], rtol=1e-12, atol=0.0)
    np.testing.assert_allclose(every.reshape(3, -1)[:, modes], a, rtol=1e-12, atol=0.0)
    errm = rel_err(mixed.reshape(3, -1)[:, modes], a)
    print(f"LiCoO2 10x10x6 full size, 3 T: mixed vs FP64 {errm:.2e}")
    assert errm <= RTOL_MIXED


@pytest.mark.skipif(os.environ.get("FP_LONG_PARITY") != "1",
                    reason="the oracle needs about 15 minutes per mode on 16 cores; set FP_LONG_PARITY=1")
@pytest.mark.parametrize("wl", [4, 5])
def test_fp64_against_the_oracle_on_the_multi_temperature_workloads(lib, wl):
    """FP64 (and double-float) rates of LiCoO2 10x10x6 (3 T) and diamond 16^3 (8 T) at full size against the oracle
    on the lowest-frequency non-degenerate mode, with the full partner sums of Eq. tao0."""
    cr = synth.workload(wl)
    w, e, v = oracle_modes(cr)
    nb = cr.nb
    flat = np.asarray(w).reshape(-1)

    def nondegenerate(m):
        q, j = divmod(m, nb)
        others = np.delete(np.asarray(w)[q], j)
        return flat[m] > 0 and np.min(np.abs(others - flat[m])) > 1e-6 * max(1.0, flat[m])

    mode = min((m for m in range(flat.size) if nondegenerate(m)), key=lambda m: flat[m])
    mask = np.zeros(flat.size, np.uint8)
    mask[mode] = 1
    with lib.Context.from_crystal(cr) as ctx:
        ctx.set_modes(w, e, v)
        r64, _ = ctx.rates4(cr.temps, cr.scalebroad, mode_mask=mask)
        rdf, _ = ctx.rates4(cr.temps, cr.scalebroad, mode_mask=mask, precision=FP_PREC_DOUBLE_FLOAT)
    nT = len(cr.temps)
    ref, _ = oracle.rates4(cr, w, e, v, sel=[mode], nthreads=CORES)
    err64 = rel_err(r64.reshape(nT, -1)[:, mode], ref[:, 0])
    errdf = rel_err(rdf.reshape(nT, -1)[:, mode], ref[:, 0])
    print(f"{cr.name}: mode {mode}, FP64 {err64:.2e}, double-float {errdf:.2e}")
    assert err64 <= RTOL_FP64 and errdf <= RTOL_FP64
