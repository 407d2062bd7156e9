"""Resumable rate sets: one long four-phonon rate set run as slices, with one checkpoint file per finished slice.

The rate of a mode is a sum over its own partners (Eq. tao0), so the rates of different q-points are independent
and a rate set splits exactly into slices of q-points.  A slice is a set of whole pairs {q, -q}, because time
reversal evaluates each pair once; the pairs are dealt to slices by equal count or by estimated cost
(sharding.balanced_shard).  Each slice is one fp_rates4 call with the mode mask of its q-points.

Checkpoints live in one directory:
* manifest.json fixes the run: grid, branch count, temperatures, broadening scale, rate options and the slice
  plan.  A rerun whose manifest differs is refused, so finished slices are never mixed with other settings.
* slice_<k>.npz holds a finished slice's rates and accepted counts.  It is written to a temporary name and then
  renamed, so a run that stops in the middle of a write leaves no file that passes for a finished slice.

A rerun loads the finished slices and computes only the others.  The assembled rates equal those of the
uninterrupted sliced run bit for bit (each slice's output is zero outside its modes and the slices are added in
order).  They equal a single whole-grid call up to the order of each mode's sum, since each slice may get a
different launch plan.
"""
from __future__ import annotations

import json
import os

import numpy as np

from .sharding import balanced_shard, rank_mask

MANIFEST = "manifest.json"


def plan_slices(grid, n_slices: int, costs=None) -> list[list[int]]:
    """q-points of each slice: the pairs {q, -q} dealt largest cost first to the least loaded slice (equal costs
    when `costs` is None, which deals equal pair counts)."""
    n_q = int(np.prod(grid))
    if n_slices < 1:
        raise ValueError("n_slices must be >= 1")
    c = np.ones(n_q) if costs is None else np.asarray(costs, np.float64)
    return balanced_shard(c, grid, n_slices)


def _jsonable(opts):
    out = {}
    for k, v in sorted(opts.items()):
        if isinstance(v, (bool, int, float, str)) or v is None:
            out[k] = v
        elif isinstance(v, np.generic):
            out[k] = v.item()
        else:
            raise ValueError(f"option {k} cannot be recorded in the manifest")
    return out


def _manifest(ctx, temps, scalebroad, opts, plan):
    return {"grid": [int(g) for g in ctx.grid], "nb": int(ctx.nb), "temps": [float(t) for t in temps],
            "scalebroad": float(scalebroad), "opts": _jsonable(opts), "slices": [[int(q) for q in s] for s in plan]}


def _atomic_savez(path, **arrays):
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def rates4_resumable(ctx, temps, scalebroad, checkpoint_dir: str, n_slices: int, costs=None, **opts):
    """Rates (nT, N, nb) of the whole grid and summed stats, computed slice by slice with checkpoints.

    ctx: a binding.Context with its modes set (anything with .grid, .N, .nb and .rates4(temps, scalebroad,
    mode_mask=..., **opts) works).  opts: fp_rates4 options; mode_mask, q_begin and q_end are set per slice and
    must not be given.  Returns (rates, stats) with stats = {"accepted": [3], "candidates", "ms",
    "slices_computed", "slices_loaded"}.
    """
    for k in ("mode_mask", "q_begin", "q_end"):
        if k in opts:
            raise ValueError(f"{k} is set per slice")
    temps = [float(t) for t in temps]
    N, nb = int(ctx.N), int(ctx.nb)
    os.makedirs(checkpoint_dir, exist_ok=True)
    mpath = os.path.join(checkpoint_dir, MANIFEST)
    if os.path.exists(mpath):
        with open(mpath) as f:
            man = json.load(f)
        plan = man["slices"]
        want = _manifest(ctx, temps, scalebroad, opts, plan)
        # the plan on disk is the one the finished slices were computed with; costs only shape a new plan
        if man != want or len(plan) != n_slices:
            raise ValueError(f"{checkpoint_dir} holds checkpoints of another run (manifest differs)")
    else:
        plan = plan_slices(ctx.grid, n_slices, costs)
        with open(mpath + ".tmp", "w") as f:
            json.dump(_manifest(ctx, temps, scalebroad, opts, plan), f)
        os.replace(mpath + ".tmp", mpath)
    rates = np.zeros((len(temps), N, nb))
    accepted = np.zeros(3)
    cands = ms = 0.0
    computed = loaded = 0
    for k, qs in enumerate(plan):
        path = os.path.join(checkpoint_dir, f"slice_{k:04d}.npz")
        if os.path.exists(path):
            with np.load(path) as z:
                r, acc, cand, t = z["rates"], z["accepted"], float(z["candidates"]), float(z["ms"])
            loaded += 1
        else:
            r, st = ctx.rates4(temps, scalebroad, mode_mask=rank_mask(qs, N, nb), **opts)
            r = np.asarray(r, np.float64).reshape(len(temps), N, nb)
            acc, cand, t = np.asarray(st["accepted"], np.float64), float(st["candidates"]), float(st["ms"])
            _atomic_savez(path, rates=r, accepted=acc, candidates=np.float64(cand), ms=np.float64(t))
            computed += 1
        rates += r
        accepted += acc
        cands += cand
        ms += t
    return rates, {"accepted": accepted.tolist(), "candidates": cands, "ms": ms, "slices_computed": computed,
                   "slices_loaded": loaded}
