"""Candidate sharding across ranks (paper_1602_05510_b300.sharding), CPU
only: the ranges of every (rank, step) are disjoint and cover the index
space, and the end-of-run reduction gives the max time and the summed
count -- checked with two gloo processes, the same collective calls the
GPU benchmark makes over NCCL."""
import os
import socket

import numpy as np
import pytest

from paper_1602_05510_b300.sharding import rank_first, reduce_timing


@pytest.mark.parametrize("world,per,steps", [(1, 5, 4), (2, 3, 5), (4, 7, 3), (8, 65536, 2)])
def test_ranges_disjoint_and_covering(world, per, steps):
    seen = np.zeros(world * per * steps, np.int32)
    for s in range(steps):
        for r in range(world):
            f = rank_first(r, world, per, s)
            seen[f:f + per] += 1
    assert (seen == 1).all()


def test_single_rank_reduction_is_identity():
    assert reduce_timing(1.5, 7, 1) == (1.5, 7)
    with pytest.raises(ValueError):
        rank_first(2, 2, 10, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        per, steps = 6, 3
        mine = [rank_first(rank, world, per, s) for s in range(steps)]
        gathered = [torch.zeros(steps, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(gathered, torch.tensor(mine, dtype=torch.int64))
        firsts = sorted(int(x) for g in gathered for x in g)
        # every block starts where the previous ends: disjoint and covering
        ok_ranges = firsts == list(range(0, world * per * steps, per))
        t, c = reduce_timing(0.25 * (rank + 1), 100 + rank, world)
        out[rank] = (ok_ranges, t, c)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        ok, t, c = res[r]
        assert ok and t == 0.5 and c == 201
