"""The N > 1 path on CPU: world_size-2 gloo ranks shard the q-grid, time with a max over
ranks and gather rates; the gathered rates equal the single-process result (oracle rates,
since no GPU is involved)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2104_04895_gb300.sharding import shard


def test_shards_cover_the_grid_once():
    for n in (1, 7, 64, 512, 4096):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                b, e = shard(n, world, r)
                assert 0 <= b <= e <= n
                seen.extend(range(b, e))
            assert seen == list(range(n))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import oracle.modes as om
    from paper_2104_04895_gb300 import synth
    from paper_2104_04895_gb300.sharding import gather_rates, max_over_ranks, shard as sh
    cr = synth.simple_cubic((3, 3, 2))
    w, e, v = om.modes(cr)
    b, en = sh(cr.nq, world, rank)
    sel = np.arange(b * cr.nb, en * cr.nb)
    r, _ = oracle.rates4(cr, w, e, v, sel=sel, nthreads=1)
    local = r.reshape(1, en - b, cr.nb)
    full = gather_rates(local, b, en, cr.nq, cr.nb, dist)
    t = max_over_ranks(float(rank + 1), dist)
    if rank == 0:
        np.save(out_path, full)
        np.save(out_path + ".t.npy", np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_shard_and_gather(tmp_path):
    out = str(tmp_path / "full.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    full = np.load(out)
    t = np.load(out + ".t.npy")
    assert t[0] == 2.0
    import oracle
    import oracle.modes as om
    from paper_2104_04895_gb300 import synth
    cr = synth.simple_cubic((3, 3, 2))
    w, e, v = om.modes(cr)
    ref, _ = oracle.rates4(cr, w, e, v)
    np.testing.assert_array_equal(full.reshape(1, -1), ref)


def _skewed_costs(grid, seed=9):
    """A cost per q-point, equal on each pair {q, -q}, with a heavy log-normal tail and a few very costly points
    (the shape of per-mode process counts across an acoustic-optical gap)."""
    from paper_2104_04895_gb300.sharding import neg_index
    n = int(np.prod(grid))
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.lognormal(0.0, 1.2, size=n)
    c[rng.choice(n, size=4, replace=False)] *= 40.0
    for q in range(n):
        c[neg_index(grid, q)] = c[min(q, neg_index(grid, q))]
    return c


def _balanced_worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import oracle.modes as om
    from paper_2104_04895_gb300 import synth
    from paper_2104_04895_gb300.sharding import balanced_shard, gather_full, load_imbalance, neg_index
    # the partitioner on a skewed cost vector of a 12^3 grid, computed independently on every rank
    g12 = (12, 12, 12)
    costs = _skewed_costs(g12)
    parts = balanced_shard(costs, g12, world)
    width = 12 ** 3  # gloo gathers equal sizes: pad each rank's list with -1
    mine = torch.full((width,), -1, dtype=torch.int64)
    mine[:len(parts[rank])] = torch.tensor(parts[rank], dtype=torch.int64)
    padded = [torch.zeros(width, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(padded, mine)
    got = [p[p >= 0] for p in padded]
    # every rank evaluates its own q-points of a small crystal (oracle rates), then one gather
    cr = synth.simple_cubic((3, 3, 2))
    w, e, v = om.modes(cr)
    small = balanced_shard(np.ones(cr.nq), cr.grid, world)
    sel = [q * cr.nb + j for q in small[rank] for j in range(cr.nb)]
    full = np.zeros((1, cr.nq, cr.nb))
    if sel:
        r, _ = oracle.rates4(cr, w, e, v, sel=sel, nthreads=1)
        full.reshape(1, -1)[:, sel] = r
    gathered = gather_full(full, dist)
    if rank == 0:
        np.save(out_path, gathered)
        np.save(out_path + ".parts.npy", np.array([load_imbalance(costs, [g.tolist() for g in got], g12),
                                                    float(sum(len(g) for g in got)),
                                                    float(all(g.tolist() == parts[i] for i, g in enumerate(got)))]))
        pairs_split = any(neg_index(g12, q) not in set(got[i].tolist()) for i in range(world) for q in got[i].tolist())
        np.save(out_path + ".split.npy", np.array([float(pairs_split)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_balanced_partition(tmp_path):
    """Two gloo ranks deal the pairs {q, -q} of a 12^3 grid by a skewed cost: both compute the same partition,
    it covers the grid once with no pair split across ranks, the heavier rank carries at most 1.1x the mean, and
    rates evaluated per rank and gathered once equal the single-process result."""
    out = str(tmp_path / "bal.npy")
    mp.spawn(_balanced_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    imb, total, same = np.load(out + ".parts.npy")
    assert same == 1.0 and total == 12 ** 3 and imb <= 1.1
    assert np.load(out + ".split.npy")[0] == 0.0
    import oracle
    import oracle.modes as om
    from paper_2104_04895_gb300 import synth
    cr = synth.simple_cubic((3, 3, 2))
    w, e, v = om.modes(cr)
    ref, _ = oracle.rates4(cr, w, e, v)
    np.testing.assert_array_equal(np.load(out).reshape(1, -1), ref)


def test_balanced_shard_beats_contiguous_ranges():
    """On the skewed costs the contiguous equal-length ranges leave one rank far above the mean; the balanced
    partition holds 1.1 for 2, 4 and 8 ranks."""
    from paper_2104_04895_gb300.sharding import balanced_shard, load_imbalance, shard
    g = (12, 12, 12)
    c = _skewed_costs(g)
    for world in (2, 4, 8):
        parts = balanced_shard(c, g, world)
        assert sorted(q for p in parts for q in p) == list(range(12 ** 3))
        assert load_imbalance(c, parts, g) <= 1.1
    contiguous = [list(range(*shard(12 ** 3, 8, r))) for r in range(8)]
    loads = [sum(c[q] for q in p) for p in contiguous]
    assert max(loads) / np.mean(loads) > 1.1


def test_cost_estimate_adds_a_common_share():
    """estimate_costs: each q-point's accepted terms from one screening pass (here a stand-in context), plus a part
    that every q-point pays alike, set to the given share of the mean cost; the q' stride defaults to N / 32."""
    from paper_2104_04895_gb300.sharding import estimate_costs

    class Ctx:
        N, nb = 64, 3

        def __init__(self, counts):
            self.counts, self.calls = counts, []

        def phase_space4(self, temps, scalebroad, stride=1, precision=0):
            self.calls.append((list(temps), scalebroad, stride))
            return self.counts, None, None

    rng = np.random.Generator(np.random.PCG64(3))
    counts = rng.integers(0, 1000, size=Ctx.N * Ctx.nb).astype(float)
    ctx = Ctx(counts)
    c = estimate_costs(ctx, [300.0, 600.0], 1.0, fixed_share=0.4)
    per_q = counts.reshape(Ctx.N, Ctx.nb).sum(axis=1)
    fixed = c - per_q
    assert np.allclose(fixed, fixed[0]) and fixed[0] > 0
    assert abs(fixed[0] / c.mean() - 0.4) < 1e-12
    assert ctx.calls == [([300.0], 1.0, 2)]        # one temperature, stride N / 32
    zero = estimate_costs(Ctx(np.zeros(Ctx.N * Ctx.nb)), [300.0], 1.0)
    assert np.all(zero == 1.0)                      # no counts: equal costs
