"""Candidate sharding across ranks (one process per GPU).

Candidates are independent, so the data path needs no collective: each
rank simulates its own candidate ranges, and only the timing and the
task-event count are reduced once at the end (max and sum)."""
from __future__ import annotations


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
