"""Host-side q-partition of a rate set over ranks (one process per GPU).

The rates of different q-points are independent (each needs only the replicated mode
tables and Phi4), so a rate set shards into contiguous q-ranges with no exchange in the
hot loop; each rank calls fp_rates4 with its [q_begin, q_end).  Timing takes the maximum
over ranks; results, when a caller wants them in one place, are gathered once at the end.
"""
from __future__ import annotations


def shard(n_q: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous q-range [begin, end) of `rank` among `world` ranks (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return (n_q * rank) // world, (n_q * (rank + 1)) // world


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
    import numpy as np
    local = np.asarray(local)
    nT = local.shape[0]
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        out = np.zeros((nT, n_q, nb))
        out[:, q_begin:q_end] = local
        return out
    import torch
    world = dist.get_world_size()
    full = torch.zeros((nT, n_q, nb), dtype=torch.float64)
    full[:, q_begin:q_end] = torch.from_numpy(np.ascontiguousarray(local))
    dist.all_reduce(full, op=dist.ReduceOp.SUM)   # ranges are disjoint, so the sum is a gather
    _ = world
    return full.numpy()
