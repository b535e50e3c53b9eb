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


# ---- the exchange step of a sharded search, with the oracle simulating each
# rank's shard of the exhaustive 3 x 3-tile search (1,024 partitions, 4 CPU +
# 1 GPU-type processors)


def test_best_pair_ties_and_empty():
    from paper_1602_05510_b300.sharding import NONE, best_pair
    assert best_pair([(5, 9), (5, 3), (7, 0)]) == (5, 3)
    assert best_pair([(NONE, -1), (8, 100)]) == (8, 100)
    assert best_pair([(NONE, -1), (NONE, -1)]) == (NONE, -1)


def _shard_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_1602_05510_b300 import workloads as W
    from paper_1602_05510_b300.sharding import NONE, gather_makespans, global_best

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        per = 1024 // world
        first = rank_first(rank, world, per, 0)
        lv = W.exhaustive_levels(10)[first:first + per]
        pl = O.make_platform(W.PLATFORMS["cfg0"])
        ms, st, _ = O.simulate_many(pl, 3, 1024, lv, threads=1)
        ok = st == 0
        if ok.any():
            m = int(ms[ok].min())
            i = first + int(np.flatnonzero(ok & (ms == m))[0])
        else:
            m, i = NONE, -1
        best = global_best(m, i, world)
        allms = gather_makespans(torch.from_numpy(ms.astype(np.int64)), world).numpy()
        out[rank] = (best, allms.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_search_equals_single_rank(world):
    """Each gloo rank runs the oracle on its own shard; the gathered
    makespans equal the single-rank run element by element, and the
    all-ranks best (makespan, lowest index) equals its argmin."""
    import torch.multiprocessing as mp

    import oracle as O
    from paper_1602_05510_b300 import workloads as W

    lv = W.exhaustive_levels(10)
    ms, st, _ = O.simulate_many(O.make_platform(W.PLATFORMS["cfg0"]), 3, 1024, lv, threads=1)
    assert (st == 0).all()
    want = (int(ms.min()), int(np.argmin(ms)))
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == set(range(world))
    for r in range(world):
        best, allms = res[r]
        assert tuple(best) == want
        assert np.array_equal(np.asarray(allms, np.int64), ms)
