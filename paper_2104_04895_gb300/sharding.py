"""Host-side partition of a rate set over ranks (one process per GPU).

The rates of different q-points are independent (each needs only the replicated mode tables and Phi4), so a rate
set shards over ranks with no exchange in the hot loop; timing takes the maximum over ranks and results, when a
caller wants them in one place, are gathered once at the end.

Two partitions:
* shard(): contiguous q-ranges of equal length (a rank passes q_begin, q_end to fp_rates4);
* balanced_shard(): the pairs {q, -q} that time reversal evaluates once, dealt to ranks by estimated cost
  (largest first to the least loaded rank), so that the uneven number of energy-conserving processes per mode
  (very uneven on the BAs-like gap, Sec. 3) does not leave one rank with most of the work.  A rank passes the mode
  mask of its q-points (rank_mask) to fp_rates4.  estimate_costs() gives the costs from a cheap pass of the rate
  kernel's screening (fp_phase_space4 on a q' stride).
"""
from __future__ import annotations

import numpy as np


def shard(n_q: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous q-range [begin, end) of `rank` among `world` ranks (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return (n_q * rank) // world, (n_q * (rank + 1)) // world


def neg_index(grid, q: int) -> int:
    """Grid index of -q (componentwise (N_a - g_a) mod N_a)."""
    g = np.unravel_index(int(q), tuple(grid))
    return int(np.ravel_multi_index(tuple((-np.asarray(g)) % np.asarray(grid)), tuple(grid)))


def pair_units(grid) -> list[tuple[int, ...]]:
    """The pairs {q, -q} of the grid (a single point where q = -q), each as a sorted tuple, by smallest index."""
    n = int(np.prod(grid))
    seen = np.zeros(n, bool)
    units = []
    for q in range(n):
        if seen[q]:
            continue
        m = neg_index(grid, q)
        seen[q] = seen[m] = True
        units.append((q,) if m == q else (q, m))
    return units


def balanced_shard(costs, grid, world: int) -> list[list[int]]:
    """q-points of each rank: the pairs {q, -q}, each costing costs[q] (one evaluation serves the pair), dealt
    largest first to the least loaded rank (ties: lower pair index, lower rank).  The result depends only on the
    arguments, so every rank computes the same partition."""
    if world < 1:
        raise ValueError("bad world size")
    costs = np.asarray(costs, np.float64).reshape(-1)
    units = pair_units(grid)
    if costs.size != int(np.prod(grid)) or np.any(~np.isfinite(costs)) or np.any(costs < 0):
        raise ValueError("costs must be N finite non-negative numbers")
    order = sorted(range(len(units)), key=lambda u: (-costs[units[u][0]], u))
    load = np.zeros(world)
    out = [[] for _ in range(world)]
    for u in order:
        r = int(np.argmin(load))
        load[r] += costs[units[u][0]]
        out[r].extend(units[u])
    return [sorted(x) for x in out]


def load_imbalance(costs, parts, grid) -> float:
    """max over ranks of the evaluated cost divided by its mean (1 = perfect); a pair {q, -q} counts once, at its
    smaller index."""
    costs = np.asarray(costs, np.float64).reshape(-1)
    loads = [sum(costs[q] for q in qs if q <= neg_index(grid, q)) for qs in parts]
    mean = float(np.mean(loads))
    return float(max(loads) / mean) if mean > 0 else 1.0


def rank_mask(qs, n_q: int, nb: int) -> np.ndarray:
    """Mode mask (N * nb bytes) selecting every branch of the q-points qs."""
    m = np.zeros((n_q, nb), np.uint8)
    m[list(qs)] = 1
    return m.reshape(-1)


def estimate_costs(ctx, temps, scalebroad, stride: int | None = None, fixed_share: float = 0.4):
    """Per-q cost estimates from one cheap pass of the rate kernel's screening: the accepted process terms of each
    q-point's modes over every stride-th q' (fp_phase_space4, mixed precision; exact decisions), plus a part that
    every q-point pays alike (assembly, contraction and screening of all pairs), set so that it is `fixed_share` of
    the mean cost."""
    from .binding import FP_PREC_MIXED
    n_q, nb = ctx.N, ctx.nb
    s = stride or max(1, n_q // 32)
    npr, _, _ = ctx.phase_space4(list(temps)[:1], scalebroad, stride=s, precision=FP_PREC_MIXED)
    acc = npr.reshape(n_q, nb).sum(axis=1)
    mean = float(acc.mean()) if acc.size else 0.0
    fixed = mean * fixed_share / (1.0 - fixed_share) if mean > 0 else 1.0
    return acc + fixed


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar (e.g. elapsed seconds) over the default process group."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rates(local, q_begin: int, q_end: int, n_q: int, nb: int, dist=None):
    """Assemble per-rank rate blocks [nT][q_begin:q_end][nb] into the full [nT][N][nb] array on every rank."""
    local = np.asarray(local)
    full = np.zeros((local.shape[0], n_q, nb))
    full[:, q_begin:q_end] = local
    return gather_full(full, dist)


def gather_full(full, dist=None):
    """Sum of per-rank full-size rate arrays [nT][N][nb] that are zero outside each rank's q-points (a partition,
    so the sum is a gather), on every rank."""
    full = np.asarray(full, np.float64)
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return full
    import torch
    t = torch.from_numpy(np.ascontiguousarray(full))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()
