"""Oracle of HeSP's iterative partition solver (Sec. 2.1 "Iterative solver").

TEST INFRASTRUCTURE ONLY (see the package docstring): plain Python over the C
oracle's simulation, in the order the paper describes one iteration.

One iteration = a schedule stage followed by a partition stage.  The
partition is one split level per base task (the dyadic 2x2 partitions of
Sec. 2.1 "Recursive task partitioners"; a base task at level l is a task
cluster of depth l), so a move changes one base task's level by one:

* Stage (1), task selection, builds the candidate list:
  - All: every base task;
  - CP: the base tasks that hold a task of the critical path of the last
    schedule -- the longest path of the DAG weighted by the scheduled
    durations (finish - start); a task is on it when the longest path
    through it is as long as the longest path overall;
  - Shallow: the base tasks whose depth (level) is minimal.
  Each selected base task below the deepest level is a candidate to be
  partitioned (level + 1); every existing task cluster (level > 0) is a
  candidate to be merged back (level - 1).  Moves are numbered
  k = 2 t + (0 partition, 1 merge) and listed in increasing k.
* Score of a move = makespan of the current partition - makespan after the
  move.  The paper estimates the latter from the parallelism available at
  the task's scheduling time; here it is the exact simulated makespan of the
  moved partition.  Only moves with a positive score are kept.
* Stage (2), sampling type: Hard takes the largest score (ties to the lower
  k); Soft draws r = floor(u * S / 2^64), S = sum of the kept scores and u the
  SplitMix64 value for counter (c = iteration, k = 0) under the solver seed,
  and takes the first kept move (in increasing k) whose running score sum
  exceeds r, i.e. each with probability score / S.
* No kept move: the partition is a local optimum and the solver stops.

With factors=True the partition is one partition factor k per base task
(one-level k-way partitions, the partition parameter p = 1/k of Sec. 2.1):
a finer move k + 1 for each selected base task below the largest factor, a
coarser move k - 1 for every base task above 1 (k = 1 merges the cluster
back); Shallow selects the base tasks with the smallest factor.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import deps, deps_side, expand, factors_to_code, lcm_of, levels_to_code, simulate, simulate_factors

MODE_ALL, MODE_CP, MODE_SHALLOW = 0, 1, 2
PICK_HARD, PICK_SOFT = 0, 1

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _sm64(seed: int, c: int, k: int) -> int:
    """SplitMix64 (Steele, Lea, Flood 2014) output for counter (c, k)."""
    z = (seed + (((c << 32) + k + 1) * _GAMMA)) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def critical_bases(pl, n: int, b: int, levels, factors: bool = False) -> tuple:
    """Schedule stage: simulate the partition and flag, per base task,
    whether one of its tasks lies on the critical path.  Returns
    (flags int8[n_base], makespan)."""
    lv = np.ascontiguousarray(levels, np.int8)
    r = simulate_factors(pl, n, b, lv) if factors else simulate(pl, n, b, lv)
    if r["status"] != 0:
        raise ValueError("simulation failed (%d)" % r["status"])
    code = factors_to_code(n, lv) if factors else levels_to_code(n, lv)
    d = expand(n, b, code)
    po, pv, _ = deps_side(n, b, code, b // lcm_of(lv)) if factors else deps(n, b, code, 1, int(lv.max()))
    T = r["n_tasks"]
    dur = [int(r["finish"][j] - r["start"][j]) for j in range(T)]
    preds = [[int(pv[e]) for e in range(po[j], po[j + 1])] for j in range(T)]
    succs = [[] for _ in range(T)]
    for j in range(T):
        for p in preds[j]:
            succs[p].append(j)
    up = [0] * T    # longest path from a source to j, including j
    for j in range(T):
        up[j] = dur[j] + max((up[p] for p in preds[j]), default=0)
    down = [0] * T  # longest path from j to a sink, including j
    for j in range(T - 1, -1, -1):
        down[j] = dur[j] + max((down[s] for s in succs[j]), default=0)
    longest = max(down)
    flags = np.zeros(len(lv), np.int8)
    for j in range(T):
        if up[j] + down[j] - dur[j] == longest:
            flags[int(d["base"][j])] = 1
    return flags, r["makespan"]


def neighbours(levels, n_levels: int, mode: int, crit=None, factors: bool = False):
    """Stage (1): the moves (k, moved levels) in increasing k.  Values lie in
    0 .. n_levels - 1 (levels) or 1 .. n_levels (factors)."""
    lo, hi = (1, n_levels) if factors else (0, n_levels - 1)
    lv = [int(x) for x in levels]
    nb = len(lv)
    if mode == MODE_ALL:
        sel = set(range(nb))
    elif mode == MODE_CP:
        sel = {t for t in range(nb) if crit[t]}
    elif mode == MODE_SHALLOW:
        m = min(lv)
        sel = {t for t in range(nb) if lv[t] == m}
    else:
        raise ValueError(mode)
    out = []
    for t in range(nb):
        if t in sel and lv[t] < hi:
            w = list(lv)
            w[t] += 1
            out.append((2 * t, np.array(w, np.int8)))
        if lv[t] > lo:
            w = list(lv)
            w[t] -= 1
            out.append((2 * t + 1, np.array(w, np.int8)))
    return out


def pick(current: int, moves: List[int], makespans: List[int], how: int, seed: int, iteration: int) -> Optional[int]:
    """Stage (2): index into `moves` of the chosen move, or None."""
    kept = [(i, current - m) for i, m in enumerate(makespans) if current - m > 0]
    if not kept:
        return None
    if how == PICK_HARD:
        best = max(s for _, s in kept)
        return min(i for i, s in kept if s == best)
    S = sum(s for _, s in kept)
    r = (_sm64(seed, iteration, 0) * S) >> 64
    run = 0
    for i, s in kept:
        run += s
        if run > r:
            return i
    raise AssertionError("unreachable")


@dataclass
class Step:
    levels: np.ndarray
    makespan: int
    moves: List[int] = field(default_factory=list)
    makespans: List[int] = field(default_factory=list)
    chosen: Optional[int] = None  # move code k, or None at a local optimum


def solve(pl, n: int, b: int, levels0, n_levels: int, mode: int, how: int, seed: int, iterations: int,
          factors: bool = False) -> List[Step]:
    """Run the iterative solver from levels0 for at most `iterations`
    iterations; one Step per iteration (the last one may be the local
    optimum where no move is kept)."""
    lv = np.ascontiguousarray(levels0, np.int8).copy()
    steps = []
    for it in range(iterations):
        crit, m = critical_bases(pl, n, b, lv, factors)
        nbrs = neighbours(lv, n_levels, mode, crit, factors)
        ms = []
        for _, w in nbrs:
            r = simulate_factors(pl, n, b, w, schedule=False) if factors else simulate(pl, n, b, w, schedule=False)
            if r["status"] != 0:
                raise ValueError("simulation failed (%d)" % r["status"])
            ms.append(r["makespan"])
        i = pick(m, [k for k, _ in nbrs], ms, how, seed, it)
        steps.append(Step(lv.copy(), m, [k for k, _ in nbrs], ms, None if i is None else nbrs[i][0]))
        if i is None:
            break
        lv = nbrs[i][1].copy()
    return steps
