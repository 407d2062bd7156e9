#!/usr/bin/env python
"""Benchmark: four-phonon process-terms/s for one full-grid RTA rate set on GB300.

Workload (default): diamond Si-like crystal, 2 atoms (nb = 6), 8x8x8 q-grid, T = 300 K,
scalebroad 1.0 -- the configuration the headline metric is quoted on.  A step is one
full-grid rate set: Bose weights, the fused persistent rate kernel (vertex assembly,
contraction, window, Gaussian, accumulation) and the fixed-order reduction.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|df|mixed] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is candidate process terms per second with the
modes resident in HBM; `e2e` is the same metric through the public C-ABI calls with host
buffers (fp_init + fp_modes + fp_rates4 + fp_free per step); `cpu_baseline` is the FP64
oracle timed on a bounded sample of the same workload on the host cores.  The same line
times the other paths on this workload (`other_precision`, `double_float`,
`mixed_tensor_cores`, `three_phonon`) and, in `configs`, the other workloads: simple cubic
4^3, zincblende BAs 12^3 (FP64 and mixed on the full grid), LiCoO2 10x10x6 with 3
temperatures and diamond 16^3 with 8 (strided q-slices where a full set would exceed
--budget-s, labelled as extrapolated), each with its error against the oracle on sampled
modes.  --surrogate, --sweep and --configs print studies instead of the bench line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2104_04895_gb300 import synth  # noqa: E402
from paper_2104_04895_gb300.sharding import (balanced_shard, estimate_costs, load_imbalance,  # noqa: E402
                                              max_over_ranks, rank_mask)

# issue rates of the two ALU pipes per SM and clock on sm_103 (GB300): 2 FP64 FMA, 128 FP32 FMA
DFMA_PER_CLK_SM = 2
FFMA_PER_CLK_SM = 128
FLOPS_PER_ACCEPTED_TERM = 25.0  # Gaussian, Bose weights and |W|^2 of one accepted term at one temperature


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["fp64", "df", "mixed"], default="fp64",
                   help="main line: fp64, df (FP64 path with its vertex contraction in double-float) or mixed")
    p.add_argument("--workload", type=int, default=2)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-other", action="store_true", help="skip timing the other precision")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--surrogate", action="store_true", help="learned-rate study instead of the bench line")
    p.add_argument("--sweep", action="store_true",
                   help="learned rates at new temperatures (36 temperatures, 3 anchors) instead of the bench line")
    p.add_argument("--configs", action="store_true",
                   help="per-workload study: time and oracle error of both precisions on workloads 1-5")
    p.add_argument("--budget-s", type=float, default=240.0,
                   help="per-workload records: a precision whose full rate set is estimated above this many seconds "
                        "is timed on strided q-slices and extrapolated")
    p.add_argument("--no-configs", action="store_true",
                   help="leave out the per-workload records (simple cubic 4^3, BAs 12^3, LiCoO2, diamond 16^3)")
    p.add_argument("--seed", type=int, default=2104)
    p.add_argument("--grid", type=int, nargs=3, default=None,
                   help="override the workload's q-grid (small profiling cases only; not a bench line)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index  # -1: do not sample
        self.proc = None
        self.lines = []

    def __enter__(self):
        if self.dev < 0:
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def alu_peaks(torch, device_index):
    """FP64 and FP32 peak TFLOP/s of this GPU from its SM count and maximum SM clock (2 flops per FMA), with the
    basis as text.  The clock comes from nvidia-smi (clocks.max.sm); without it, 2070 MHz, GB300's maximum."""
    nsm = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz, src = 2070.0, "GB300 maximum SM clock"
    try:
        r = subprocess.run(["nvidia-smi", "-i", str(device_index), "--query-gpu=clocks.max.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=30)
        mhz, src = float(r.stdout.strip().splitlines()[0]), "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    fp64 = nsm * mhz * 1e6 * DFMA_PER_CLK_SM * 2 / 1e12
    fp32 = nsm * mhz * 1e6 * FFMA_PER_CLK_SM * 2 / 1e12
    basis = (f"derived: {nsm} SMs x {mhz:.0f} MHz ({src}) x {DFMA_PER_CLK_SM} DFMA or {FFMA_PER_CLK_SM} FFMA "
             f"per clock and SM x 2 flops")
    return fp64, fp32, basis


def e2e_input_bytes(binding, cr):
    """Bytes a step hands the library from host memory: the buffers passed to fp_init (lattice, positions,
    masses, the packed Phi2 and Phi4 lists), fp_set_fc3 (packed Phi3) and fp_rates4 (temperatures), measured from
    the objects themselves."""
    import ctypes
    n = np.ascontiguousarray(cr.lattice, np.float64).nbytes + np.ascontiguousarray(cr.frac, np.float64).nbytes
    n += np.ascontiguousarray(cr.mass, np.float64).nbytes + 8 * len(cr.temps)
    n += ctypes.sizeof(binding.pack_fc2(cr.fc2_idx, cr.fc2_val)) + ctypes.sizeof(binding.pack_fc4(cr.fc4_idx,
                                                                                                  cr.fc4_val))
    if cr.fc3_idx is not None:
        n += len(cr.fc3_idx) * ctypes.sizeof(binding.fp_fc3)
    return int(n)


def cpu_baseline(cr, seconds, w=None, e=None, v=None):
    """FP64 oracle on sampled modes with full partner sums, until about `seconds` of CPU work."""
    import oracle
    import oracle.modes as om
    if w is None:
        w, e, v = om.modes(cr)
    rng = np.random.Generator(np.random.PCG64(2104))
    order = rng.permutation(np.arange(cr.nb, cr.nq * cr.nb))
    cores = os.cpu_count() or 1
    sel, ref, t_total = [], [], 0.0
    for m in order:
        t0 = time.perf_counter()
        r, _ = oracle.rates4(cr, w, e, v, sel=[int(m)], nthreads=cores)
        t_total += time.perf_counter() - t0
        sel.append(int(m))
        ref.append(r[:, 0])
        if t_total >= seconds:
            break
    cands = 3.0 * len(sel) * cr.nq ** 2 * cr.nb ** 3
    return {"value": cands / t_total, "unit": "process-terms/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(sel)} modes of {cr.name} {cr.grid[0]}x{cr.grid[1]}x{cr.grid[2]} with full (q',q'') "
                      f"partner sums, {t_total:.1f} s", "seconds": t_total}, sel, np.array(ref).T


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cr = synth.workload(args.workload)
    import oracle
    import oracle.modes as om
    w, e, v = om.modes(cr)
    cores = os.cpu_count() or 1
    rng = np.random.Generator(np.random.PCG64(7))
    order = rng.permutation(np.arange(cr.nb, cr.nq * cr.nb))
    per_step = 1
    times = []
    for s in range(args.warmup + args.steps):
        sel = [int(m) for m in order[s * per_step:(s + 1) * per_step]]
        t0 = time.perf_counter()
        oracle.rates4(cr, w, e, v, sel=sel, nthreads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    cands = 3.0 * per_step * cr.nq ** 2 * cr.nb ** 3
    val = cands * len(times) / sum(times)
    line = {"impl": "reference", "metric": "four-phonon process-terms/s", "value": val, "unit": "process-terms/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": synth.WORKLOAD_NAMES[args.workload], "sample_modes_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": "process-terms/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} mode(s) per step with full partner sums"},
            "e2e": {"value": val, "unit": "process-terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_precision(ctx, binding, torch, cr, prec, part, out, flush, stream, steps, warmup, barrier, clk=None):
    """Time `steps` full rate sets (after `warmup`) with CUDA events on the library's stream; `part` holds this
    rank's rate options (its mode mask under a multi-GPU partition)."""
    def step():
        return ctx.rates4_device(cr.temps, out.data_ptr(), cr.scalebroad, precision=prec, **part)

    for _ in range(warmup):
        st = step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kernel_ms = []
    barrier()
    torch.cuda.synchronize()
    sampler = clk if clk is not None else ClockSampler(-1)
    with sampler:
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            st = step()
            ev[i][1].record(stream)
            kernel_ms.append(st["ms"])
        torch.cuda.synchronize()
    barrier()
    return float(sum(a.elapsed_time(b) for a, b in ev)), float(np.mean(kernel_ms)), st


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.surrogate:
        return run_surrogate(args)
    if args.sweep:
        return run_sweep(args)
    if args.configs:
        return run_configs(args)
    import torch
    import torch.distributed as dist
    from paper_2104_04895_gb300 import binding

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    main_prec = {"fp64": binding.FP_PREC_FP64, "df": binding.FP_PREC_DOUBLE_FLOAT,
                 "mixed": binding.FP_PREC_MIXED}[args.precision]
    other_prec = binding.FP_PREC_FP64 if main_prec == binding.FP_PREC_MIXED else binding.FP_PREC_MIXED
    cr = synth.workload(args.workload)
    if args.grid:
        cr = cr.with_grid(args.grid)
    N, nb, nT = cr.nq, cr.nb, len(cr.temps)

    def barrier():
        if ws > 1:
            dist.barrier()

    ctx = binding.Context.from_crystal(cr, device=local)
    stream = torch.cuda.current_stream(dev)
    ctx.set_stream(stream.cuda_stream)
    w, e, v = ctx.modes()
    out = torch.zeros(nT * N * nb, dtype=torch.float64, device=dev)
    out_other = torch.zeros(nT * N * nb, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > 129 MB L2
    tuned = None
    if not args.no_autotune:
        tuned, _ = ctx.autotune(cr.temps, cr.scalebroad, precision=binding.FP_PREC_MIXED)

    cands_step = 3.0 * N * N * N * nb ** 4          # all ranks together: one full-grid rate set per step
    clk = ClockSampler(local)
    # this rank's q-points: all of them on one GPU; on several, the pairs {q, -q} dealt by estimated cost (every
    # rank computes the same integer counts, hence the same partition, with no communication)
    part, part_desc = {}, "one GPU, whole grid"
    if ws > 1:
        costs = estimate_costs(ctx, cr.temps, cr.scalebroad)
        parts = balanced_shard(costs, cr.grid, ws)
        part = {"mode_mask": rank_mask(parts[rank], N, nb)}
        part_desc = (f"pairs {{q, -q}} dealt by estimated cost over {ws} GPUs, estimated max/mean "
                     f"{load_imbalance(costs, parts, cr.grid):.3f}")
    total_ms, kms, st = time_precision(ctx, binding, torch, cr, main_prec, part, out, flush, stream, args.steps,
                                       args.warmup, barrier, clk)
    total_ms = max_over_ranks(total_ms, dist if ws > 1 else None, dev)
    value = cands_step * args.steps / (total_ms * 1e-3)
    # algorithmic flops per launch: the vertex work of this factorization (fp_stats.flops) plus the
    # accumulation of every accepted term at every temperature (Gaussian, Bose weights, |W|^2: 25 flops)
    acc_flops = FLOPS_PER_ACCEPTED_TERM * st["terms_executed"] * nT
    achieved_tflops = (st["flops"] + acc_flops) / (kms * 1e-3) / 1e12
    fp64_peak, fp32_peak, peak_basis = alu_peaks(torch, local)
    peak = fp32_peak if main_prec == binding.FP_PREC_MIXED else fp64_peak
    other = None
    if not args.no_other:
        o_ms, o_kms, o_st = time_precision(ctx, binding, torch, cr, other_prec, part, out_other, flush, stream,
                                           args.steps, args.warmup, barrier)
        o_ms = max_over_ranks(o_ms, dist if ws > 1 else None, dev)
        o_peak = fp64_peak if other_prec == binding.FP_PREC_FP64 else fp32_peak
        o_ach = (o_st["flops"] + FLOPS_PER_ACCEPTED_TERM * o_st["terms_executed"] * nT) / (o_kms * 1e-3) / 1e12
        other = {"precision": "fp64" if other_prec == binding.FP_PREC_FP64 else "mixed",
                 "value": cands_step * args.steps / (o_ms * 1e-3), "unit": "process-terms/s",
                 "s_per_rate_set": o_ms / args.steps * 1e-3, "tile": o_st["tile"],
                 "roofline": {"bound": "alu", "achieved": o_ach, "peak": o_peak, "unit": "TFLOP/s",
                              "frac": o_ach / o_peak,
                              "pipe": "fp64" if other_prec == binding.FP_PREC_FP64 else "fp32",
                              "kernel_ms": o_kms}}

    # the FP64-accurate path with its vertex contraction in double-float (when it is not the main line)
    dfl = None
    if not args.no_other and main_prec != binding.FP_PREC_DOUBLE_FLOAT:
        out_df = torch.zeros(nT * N * nb, dtype=torch.float64, device=dev)
        d_ms, d_kms, d_st = time_precision(ctx, binding, torch, cr, binding.FP_PREC_DOUBLE_FLOAT, part, out_df, flush,
                                           stream, args.steps, args.warmup, barrier)
        d_ms = max_over_ranks(d_ms, dist if ws > 1 else None, dev)
        dfl = {"precision": "fp64 path, vertex contraction in double-float on the FP32 pipes",
               "value": cands_step * args.steps / (d_ms * 1e-3), "unit": "process-terms/s",
               "s_per_rate_set": d_ms / args.steps * 1e-3, "tile": d_st["tile"], "kernel_ms": d_kms}

    # the mixed path with its per-q'' contraction T = A conj(E3) on the tensor cores (tcgen05 kind::tf32, 3xTF32)
    tensor = None
    if not args.no_other and nb == 6:
        out_tc = torch.zeros(nT * N * nb, dtype=torch.float64, device=dev)
        t_ms, t_kms, t_st = time_precision(ctx, binding, torch, cr, binding.FP_PREC_MIXED, {**part, "tensor_cores": 1},
                                           out_tc, flush, stream, args.steps, args.warmup, barrier)
        t_ms = max_over_ranks(t_ms, dist if ws > 1 else None, dev)
        tensor = {"precision": "mixed, T contraction on tcgen05 (kind::tf32, 3xTF32)",
                  "value": cands_step * args.steps / (t_ms * 1e-3), "unit": "process-terms/s",
                  "s_per_rate_set": t_ms / args.steps * 1e-3, "tile": t_st["tile"], "kernel_ms": t_kms}

    # three-phonon rates of the same workload (FP64), for context: the mean device time of `steps` rate sets
    # after `warmup`, each from CUDA events on the library's stream
    three = None
    if not args.no_other and cr.fc3_idx is not None:
        for _ in range(args.warmup):
            ctx.rates3(cr.temps, cr.scalebroad, **part)
        ms3 = []
        for _ in range(max(1, args.steps)):
            _, st3 = ctx.rates3(cr.temps, cr.scalebroad, **part)
            ms3.append(st3["ms"])
        s3 = max_over_ranks(float(np.mean(ms3)), dist if ws > 1 else None, dev) * 1e-3
        three = {"precision": "fp64", "s_per_rate_set": s3, "steps": len(ms3), "candidates": st3["candidates"],
                 "terms_per_s": st3["candidates"] / s3, "accepted": st3["accepted"][:2]}

    # end to end through the public API with host buffers
    e2e_times = []
    h2d = d2h = 0
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        with binding.Context.from_crystal(cr, device=local) as c2:
            c2.modes(copy=False)
            r, _ = c2.rates4(cr.temps, cr.scalebroad, precision=main_prec, **part, **(tuned or {}))
        t1 = time.perf_counter()
        if i > 0:
            e2e_times.append(t1 - t0)
        h2d = e2e_input_bytes(binding, cr)
        d2h = r.nbytes
    e2e_s = float(np.mean(e2e_times)) if e2e_times else float("nan")
    e2e_s = max_over_ranks(e2e_s, dist if ws > 1 else None, dev)
    e2e_value = cands_step / e2e_s

    # the other benchmark workloads, one record each (rank 0 of a single-GPU run)
    configs = None
    if ws == 1 and not args.no_configs and not args.grid:
        configs = []
        for wl in (1, 3, 4, 5):
            try:
                configs.append(measure_workload(binding, wl, full_max_s=args.budget_s,
                                                df_full_max_s=min(60.0, args.budget_s), tensor_cores=False,
                                                oracle_check=not args.no_cpu_baseline))
            except Exception as exc:  # a failed record is reported in the line; it must not cost the main line
                configs.append({"workload": synth.WORKLOAD_NAMES[wl], "error": f"{type(exc).__name__}: {exc}"})

    if rank == 0:
        base = None
        rel_err = rel_err_other = None
        # the oracle baseline and the sampled error check run at N = 1 only: with several GPUs rank 0 holds only the
        # rates of its own q-points
        if not args.no_cpu_baseline and ws == 1:
            base, sel, ref = cpu_baseline(cr, args.cpu_sample_seconds, w, e, v)
            gpu = out.view(nT, N * nb).cpu().numpy()[:, sel]
            rel_err = float(np.max(np.abs(gpu - ref) / np.abs(ref)))
            if other is not None:
                g2 = out_other.view(nT, N * nb).cpu().numpy()[:, sel]
                other["rel_err_vs_oracle_sampled"] = float(np.max(np.abs(g2 - ref) / np.abs(ref)))
            if tensor is not None:
                g3 = out_tc.view(nT, N * nb).cpu().numpy()[:, sel]
                tensor["rel_err_vs_oracle_sampled"] = float(np.max(np.abs(g3 - ref) / np.abs(ref)))
            if dfl is not None:
                g4 = out_df.view(nT, N * nb).cpu().numpy()[:, sel]
                dfl["rel_err_vs_oracle_sampled"] = float(np.max(np.abs(g4 - ref) / np.abs(ref)))
            base.pop("seconds", None)
        line = {
            "metric": "four-phonon process-terms/s", "value": value, "unit": "process-terms/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "s_per_rate_set": total_ms / args.steps * 1e-3,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": {binding.FP_PREC_FP64: "f64", binding.FP_PREC_DOUBLE_FLOAT: "f64+f32x2",
                      binding.FP_PREC_MIXED: "f32+f64"}[main_prec],
            "data": "synthetic",
            "config": {"workload": synth.WORKLOAD_NAMES[args.workload] if not args.grid else
                       f"{cr.name} {args.grid[0]}x{args.grid[1]}x{args.grid[2]} (profiling case)",
                       "precision": args.precision,
                       "candidates_per_step": cands_step, "accepted_per_step": st["accepted"],
                       "candidates_executed_per_step": st["candidates_executed"],
                       "time_reversal": "one q of each pair {q, -q} evaluated, rates written at both",
                       "l2": "flushed between timed steps (256 MB write)", "tile": st["tile"],
                       "autotuned_mixed_tile": tuned,
                       "parallelism": part_desc},
            "rel_err_vs_oracle_sampled": rel_err,
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved_tflops / peak, "traffic": None, "peak_basis": peak_basis,
                         "pipe": "fp32" if main_prec == binding.FP_PREC_MIXED else "fp64",
                         "kernel_ms": kms, "flops_per_launch": st["flops"] + acc_flops,
                         "flops_vertex": st["flops"], "flops_accumulate": acc_flops},
            "other_precision": other,
            "mixed_tensor_cores": tensor,
            "double_float": dfl,
            "three_phonon": three,
            "configs": configs,
            "cpu_baseline": base,
            "e2e": {"value": e2e_value, "unit": "process-terms/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "s_per_rate_set": e2e_s},
            "gpu_launches": 4 * args.steps,  # per timed step: Bose weights, FP32 tables, rate kernel, reduction
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def run_surrogate(args):
    """Learned rates against the exact, temperature-batched mixed path on the same workload (one JSON line).

    The exact path's time per full-grid rate set comes from three strided q-slices (as in the per-workload
    records) when a full set would exceed --budget-s, else from a full set.  The surrogate runs as specified:
    exact rates on a seeded 10 % of the pairs {q, -q} train the network, 5 % judge it per bin, bins above 5 %
    held-out error fall back to exact rates.  The error it actually makes is measured on a seeded sample of the
    entries it predicted (exact rates of 200 of those modes)."""
    import torch
    from paper_2104_04895_gb300 import binding
    cr = synth.workload(args.workload)
    if args.grid:
        cr = cr.with_grid(args.grid)
    N, nb, nT = cr.nq, cr.nb, len(cr.temps)
    cands = 3.0 * N ** 3 * nb ** 4
    full_exec = 3.0 * N * N * nb ** 3 * nb * (N + _self_conjugate(cr.grid)) / 2.0
    with binding.Context.from_crystal(cr) as ctx:
        ctx.modes(copy=False)
        ctx.autotune(cr.temps, cr.scalebroad, precision=binding.FP_PREC_MIXED)
        probe = np.zeros(N * nb, np.uint8)
        probe[nb:2 * nb] = 1
        _, st = ctx.rates4(cr.temps, cr.scalebroad, precision=binding.FP_PREC_MIXED, mode_mask=probe, no_graph=1)
        est = st["ms"] * 1e-3 * full_exec / st["candidates_executed"]
        if est <= args.budget_s:
            _, st = ctx.rates4(cr.temps, cr.scalebroad, precision=binding.FP_PREC_MIXED)
            t_exact, how = st["ms"] * 1e-3, "full grid, one rate set"
        else:
            m = max(2, int(np.ceil(N * est / ((N + _self_conjugate(cr.grid)) / 2.0) / 20.0)))
            ext = []
            for k in (0, m // 3, (2 * m) // 3):
                _, st = ctx.rates4(cr.temps, cr.scalebroad, precision=binding.FP_PREC_MIXED,
                                   mode_mask=_slice_mask(cr, m, k), no_graph=1)
                ext.append(st["ms"] * 1e-3 * full_exec / st["candidates_executed"])
            t_exact, how = float(np.mean(ext)), f"extrapolated from three strided q-slices (q = k mod {m})"
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.surrogate_fit(cr.temps, cr.scalebroad, seed=args.seed)
        t_sur = time.perf_counter() - t0
        rates, used = ctx.surrogate_rates()
        pred_modes = np.nonzero(((used == 0) & (rates > 0)).any(axis=0).reshape(-1))[0]
        rel = np.array([])
        if pred_modes.size:
            rng = np.random.Generator(np.random.PCG64(args.seed + 1))
            pick = np.sort(rng.choice(pred_modes, size=min(200, pred_modes.size), replace=False))
            mask = np.zeros(N * nb, np.uint8)
            mask[pick] = 1
            ex, _ = ctx.rates4(cr.temps, cr.scalebroad, precision=binding.FP_PREC_MIXED, mode_mask=mask, no_graph=1)
            ex = ex.reshape(nT, -1)[:, pick]
            pr = rates.reshape(nT, -1)[:, pick]
            ok = ex > 0
            rel = np.abs(pr[ok] - ex[ok]) / ex[ok]
    pos = rates > 0
    line = {"metric": "four-phonon rate set: surrogate vs exact (mixed, temperature-batched)",
            "workload": synth.WORKLOAD_NAMES.get(args.workload) if not args.grid else
            f"{cr.name} {args.grid[0]}x{args.grid[1]}x{args.grid[2]} T={list(cr.temps)}",
            "exact_mixed_s": t_exact, "exact_timing": how, "exact_terms_per_s": cands / t_exact,
            "surrogate_s": t_sur, "speedup": t_exact / t_sur,
            "exact_share": float(used[pos].mean()), "predicted_modes": int(pred_modes.size),
            "predicted_rel_err_sampled": {"n": int(rel.size),
                                          "median": float(np.median(rel)) if rel.size else None,
                                          "p90": float(np.quantile(rel, 0.9)) if rel.size else None,
                                          "max": float(rel.max()) if rel.size else None},
            "report": rep}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """Learned rates at new temperatures against the exact path (one JSON line).

    Output temperatures 300..1000 K every 20 K (36): the exact path needs five temperature-batched rate sets (8, 8,
    8, 8, 4 temperatures), each timed here on strided q-slices of the grid (or in full when it is short).  The
    surrogate takes exact rates of every mode at 300, 650 and 1000 K (one batched set) and of a seeded 15 % of the
    pairs {q, -q} at the 36 temperatures, trains, predicts and falls back per bin.  Its realised error is measured
    on exact rates of a seeded sample of 200 predicted modes at all 36 temperatures."""
    from paper_2104_04895_gb300 import binding
    cr = synth.workload(args.workload)
    if args.grid:
        cr = cr.with_grid(args.grid)
    N, nb = cr.nq, cr.nb
    temps = [float(t) for t in np.arange(300.0, 1000.0 + 1e-9, 20.0)]
    anchors = [300.0, 650.0, 1000.0]
    full_exec = 3.0 * N * N * nb ** 3 * nb * (N + _self_conjugate(cr.grid)) / 2.0
    prec = binding.FP_PREC_MIXED
    with binding.Context.from_crystal(cr) as ctx:
        ctx.modes(copy=False)
        ctx.autotune(temps[:8], cr.scalebroad, precision=prec)
        t_exact, parts = 0.0, []
        for i in range(0, len(temps), 8):
            chunk = temps[i:i + 8]
            probe = np.zeros(N * nb, np.uint8)
            probe[nb:2 * nb] = 1
            _, st = ctx.rates4(chunk, cr.scalebroad, precision=prec, mode_mask=probe, no_graph=1)
            est = st["ms"] * 1e-3 * full_exec / st["candidates_executed"]
            if est <= args.budget_s:
                _, st = ctx.rates4(chunk, cr.scalebroad, precision=prec)
                secs = st["ms"] * 1e-3
            else:
                m = max(2, int(np.ceil(N * est / ((N + _self_conjugate(cr.grid)) / 2.0) / 20.0)))
                ext = []
                for k in (0, m // 3, (2 * m) // 3):
                    _, st = ctx.rates4(chunk, cr.scalebroad, precision=prec, mode_mask=_slice_mask(cr, m, k),
                                       no_graph=1)
                    ext.append(st["ms"] * 1e-3 * full_exec / st["candidates_executed"])
                secs = float(np.mean(ext))
            parts.append(secs)
            t_exact += secs
        t0 = time.perf_counter()
        rates, used, rep = ctx.surrogate_sweep(anchors, temps, cr.scalebroad, seed=args.seed)
        t_sur = time.perf_counter() - t0
        pred_modes = np.nonzero(((used == 0) & (rates > 0)).any(axis=0).reshape(-1))[0]
        rel = np.array([])
        if pred_modes.size:
            rng = np.random.Generator(np.random.PCG64(args.seed + 1))
            pick = np.sort(rng.choice(pred_modes, size=min(200, pred_modes.size), replace=False))
            mask = np.zeros(N * nb, np.uint8)
            mask[pick] = 1
            ex = np.concatenate([ctx.rates4(temps[i:i + 8], cr.scalebroad, precision=prec, mode_mask=mask,
                                            no_graph=1)[0].reshape(-1, N * nb)[:, pick] for i in range(0, len(temps), 8)])
            pr = rates.reshape(len(temps), -1)[:, pick]
            ok = (ex > 0) & (used.reshape(len(temps), -1)[:, pick] == 0)
            rel = np.abs(pr[ok] - ex[ok]) / ex[ok]
    pos = rates > 0
    line = {"metric": "four-phonon rates at new temperatures: surrogate vs exact (mixed, temperature-batched)",
            "workload": f"{cr.name} {cr.grid[0]}x{cr.grid[1]}x{cr.grid[2]} nb={nb}",
            "temperatures": len(temps), "anchors": anchors,
            "exact_s": t_exact, "exact_batches_s": parts, "surrogate_s": t_sur, "speedup": t_exact / t_sur,
            "exact_share": float(used[pos].mean()), "predicted_modes": int(pred_modes.size),
            "predicted_rel_err_sampled": {"n": int(rel.size), "median": float(np.median(rel)) if rel.size else None,
                                          "p90": float(np.quantile(rel, 0.9)) if rel.size else None,
                                          "max": float(rel.max()) if rel.size else None},
            "report": rep}
    print(json.dumps(line), flush=True)


def _self_conjugate(grid):
    """Number of grid points q with -q = q (mod the grid)."""
    n = 1
    for g in grid:
        n *= 2 if g % 2 == 0 else 1
    return n


def _slice_mask(cr, m, k):
    """All branches of the q-points q = k (mod m): a strided slice that spreads over the whole grid."""
    mask = np.zeros((cr.nq, cr.nb), np.uint8)
    mask[k::m] = 1
    return mask.reshape(-1)


def measure_workload(binding, wl, budget_slice_s=10.0, full_max_s=300.0, oracle_max_s=150.0, df_full_max_s=None,
                     tensor_cores=True, oracle_check=True):
    """Seconds per full-grid rate set of workload `wl` in each precision, and errors on sampled modes.

    An FP64 or mixed rate set estimated (from a one-q probe) to stay under `full_max_s` is timed on the whole grid,
    a double-float one under `df_full_max_s` (default: the same), and the tensor-core option (nb = 6 only) when
    `tensor_cores` is set and the mixed set ran in full.  Otherwise three strided q-slices (q = k mod m, all
    branches) of about `budget_slice_s` each are timed and scaled to the grid
    by the candidates the kernel screened (time reversal evaluates (N + self-conjugate points) / 2 points of a full
    grid); the spread of the three gives the sampling uncertainty.  The rates use the library's own modes
    (fp_modes); with `oracle_check`, the oracle (the CPU-baseline leg of this record) recomputes a ruled mode sample
    (lowest positive frequency and one seeded mode) from the same mode tables, so the error is a strict one; it runs
    only where it finishes within `oracle_max_s` on the host cores."""
    cr = synth.workload(wl)
    N, nb, nT = cr.nq, cr.nb, len(cr.temps)
    cands = 3.0 * N ** 3 * nb ** 4
    full_exec = 3.0 * N * N * nb ** 3 * nb * (N + _self_conjugate(cr.grid)) / 2.0
    outs = {}
    with binding.Context.from_crystal(cr) as ctx:
        w, e, v = ctx.modes()
        flat = w.reshape(-1)
        pos = np.nonzero(flat > 0)[0]
        rng = np.random.Generator(np.random.PCG64(77 + wl))
        sample = [int(pos[np.argmin(flat[pos])]), int(rng.choice(pos))]
        if N * nb > 5000:
            sample = sample[:1]  # the oracle takes a minute or more per mode here
        res = {"workload": synth.WORKLOAD_NAMES[wl], "candidates": cands, "temperatures": nT,
               "sample_modes": sample, "modes": "fp_modes (GPU)"}
        for name, prec in (("fp64", binding.FP_PREC_FP64), ("double_float", binding.FP_PREC_DOUBLE_FLOAT),
                           ("mixed", binding.FP_PREC_MIXED)):
            probe = np.zeros(N * nb, np.uint8)
            probe[nb:2 * nb] = 1                                   # q = 1, all branches (also warms the kernel)
            _, st = ctx.rates4(cr.temps, cr.scalebroad, precision=prec, mode_mask=probe, no_graph=1)
            t_rep = st["ms"] * 1e-3 * nb * 3.0 * N * N * nb ** 3 / st["candidates_executed"]
            est = t_rep * full_exec / (nb * 3.0 * N * N * nb ** 3)
            limit = df_full_max_s if (name == "double_float" and df_full_max_s is not None) else full_max_s
            if 0.5 * limit < est < 2.0 * limit:
                # near the limit: one q is not representative (accepted counts vary over the grid); 16 spread q
                _, st = ctx.rates4(cr.temps, cr.scalebroad, precision=prec,
                                   mode_mask=_slice_mask(cr, max(1, N // 16), 1), no_graph=1)
                t_rep = st["ms"] * 1e-3 * nb * 3.0 * N * N * nb ** 3 / st["candidates_executed"]
                est = t_rep * full_exec / (nb * 3.0 * N * N * nb ** 3)
            smask = np.zeros(N * nb, np.uint8)
            smask[sample] = 1
            if est <= limit:
                out, st = ctx.rates4(cr.temps, cr.scalebroad, precision=prec)
                secs = st["ms"] * 1e-3
                rec = {"s_per_rate_set": secs, "terms_per_s": cands / secs, "timing": "full grid, one rate set",
                       "accepted": st["accepted"], "candidates_executed": st["candidates_executed"]}
                outs[name] = out.reshape(nT, -1)[:, sample]
            else:
                m = max(2, int(np.ceil(N * t_rep / budget_slice_s)))
                ext = []
                for k in (0, m // 3, (2 * m) // 3):
                    _, st = ctx.rates4(cr.temps, cr.scalebroad, precision=prec, mode_mask=_slice_mask(cr, m, k),
                                       no_graph=1)
                    ext.append(st["ms"] * 1e-3 * full_exec / st["candidates_executed"])
                secs = float(np.mean(ext))
                rec = {"s_per_rate_set": secs, "terms_per_s": cands / secs,
                       "timing": f"extrapolated from three strided q-slices (q = k mod {m}, k = 0, {m // 3}, "
                                 f"{(2 * m) // 3}) by screened candidates",
                       "slice_spread": float((max(ext) - min(ext)) / secs)}
                out, _ = ctx.rates4(cr.temps, cr.scalebroad, precision=prec, mode_mask=smask, no_graph=1)
                outs[name] = out.reshape(nT, -1)[:, sample]
            rec["tile"] = st["tile"]
            res[name] = rec
        if tensor_cores and nb == 6 and res["mixed"]["timing"].startswith("full grid"):
            out, st = ctx.rates4(cr.temps, cr.scalebroad, precision=binding.FP_PREC_MIXED, tensor_cores=1)
            secs = st["ms"] * 1e-3
            res["mixed_tensor_cores"] = {"s_per_rate_set": secs, "terms_per_s": cands / secs, "tile": st["tile"],
                                         "timing": "full grid, one rate set"}
            outs["mixed_tensor_cores"] = out.reshape(nT, -1)[:, sample]
    res["mixed"]["rel_err_vs_fp64_gpu"] = float(np.max(np.abs(outs["mixed"] - outs["fp64"]) / outs["fp64"]))
    # oracle cost per mode on these host cores: about 3 N^2 nb^3 terms at 1.6e7 (6 / nb)^3 terms/s on 16 cores
    cores = os.cpu_count() or 1
    t_or = 3.0 * N ** 2 * nb ** 3 / (1.6e7 * (6.0 / nb) ** 3 * cores / 16.0)
    if not oracle_check:
        res["oracle"] = {"skipped": "no CPU baseline in this run"}
    elif t_or * len(sample) <= oracle_max_s:
        import oracle
        t0 = time.perf_counter()
        ref, _ = oracle.rates4(cr, w, e, v, sel=sample, nthreads=cores)
        dt = time.perf_counter() - t0
        res["oracle"] = {"s_per_mode": dt / len(sample), "terms_per_s": 3.0 * N ** 2 * nb ** 3 * len(sample) / dt,
                         "cores": cores}
        for name in outs:
            res[name]["rel_err_vs_oracle"] = float(np.max(np.abs(outs[name] - ref) / ref))
    else:
        res["oracle"] = {"skipped": f"about {t_or:.0f} s per mode on {cores} cores"}
    return res


def run_configs(args):
    """One JSON line per workload (see measure_workload)."""
    from paper_2104_04895_gb300 import binding
    for wl in (1, 2, 3, 4, 5):
        print(json.dumps(measure_workload(binding, wl, full_max_s=args.budget_s)), flush=True)


if __name__ == "__main__":
    main()
