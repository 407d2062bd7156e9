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
