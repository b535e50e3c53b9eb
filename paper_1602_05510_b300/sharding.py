"""Candidate sharding across ranks (one process per GPU).

Candidates are independent, so each rank simulates its own candidate
ranges.  The result of a search step is the best partition over all ranks
(the partition stage of the iterative solver keeps the best schedule, Sec.
2.1): each rank reduces its own shard to (least makespan, lowest candidate
index at it) on its device, and `global_best` combines those pairs across
ranks with one all-gather of 16 bytes per rank.  `gather_makespans` is the
alternative exchange, every makespan (8 bytes per candidate) to every rank.
The timing and the task-event count are reduced once at the end (max and
sum)."""
from __future__ import annotations

NONE = (1 << 63) - 1  # makespan of a shard with no successful candidate


def rank_first(rank: int, world: int, per_rank: int, step: int) -> int:
    """First candidate index of `rank` at `step`: per_rank consecutive
    candidates, ranks interleaved step after step, so no two (rank, step)
    pairs share a candidate and the first world * per_rank * steps indices
    are all covered."""
    if not (0 <= rank < world) or per_rank < 0 or step < 0:
        raise ValueError("bad rank / world / step")
    return (step * world + rank) * per_rank


def reduce_timing(seconds: float, count: int, world: int, device=None):
    """(max over ranks of `seconds`, sum over ranks of `count`); a plain
    return for one rank, an all-reduce of two scalars otherwise (any
    torch.distributed backend: nccl on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(seconds), int(count)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([int(count)], dtype=torch.int64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def best_pair(pairs):
    """The least (makespan, global index) of (makespan, index) pairs, ties
    to the lower index; (NONE, -1) when no pair holds a candidate."""
    live = [(int(m), int(i)) for m, i in pairs if int(m) != NONE and int(i) >= 0]
    return min(live) if live else (NONE, -1)


def global_best(best, index, world, device=None):
    """The best candidate over every rank: `best` is this rank's least
    makespan (NONE if it has no successful candidate) and `index` the global
    index of its lowest-indexed candidate at that makespan.  Returns the
    least (makespan, index) over ranks, ties to the lower global index, the
    same answer a single rank holding every candidate would give.  A
    device tensor of two int64 may be passed instead of the two numbers (it
    is gathered without a host round trip before the collective)."""
    import torch
    if isinstance(best, torch.Tensor):
        t = best.reshape(2).to(torch.int64)
    else:
        t = torch.tensor([int(best), int(index)], dtype=torch.int64, device=device)
    if world <= 1:
        return best_pair([t.tolist()])
    import torch.distributed as dist
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    return best_pair([o.tolist() for o in out])


def gather_makespans(makespan, world):
    """Every rank's makespans (equal-sized shards), concatenated in rank
    order on every rank: 8 bytes per candidate."""
    import torch
    if world <= 1:
        return makespan
    import torch.distributed as dist
    out = [torch.empty_like(makespan) for _ in range(world)]
    dist.all_gather(out, makespan)
    return torch.cat(out)
