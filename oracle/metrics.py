"""Oracle of the Table 1 metrics (Sec. 3) and of the table's procedure.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Metrics of one simulated partition of an N x N Cholesky (N = n b):
  GFLOPS  = (N^3 / 3) / makespan (flops per ns);
  load    = busy / (P makespan), busy = the tasks' summed execution time,
            P = processors: the processors' average busy share;
  avg block = the mean block size over the tasks;
  depth   = 1 + the deepest split level (the levels of the task hierarchy).

Table procedure, per platform and scheduling policy:
  homogeneous: simulate the unsplit partition for each tile size b of the
  sweep (n = N / b tiles); the best (smallest makespan, ties to the larger
  b) gives the homogeneous columns;
  heterogeneous: from that partition, the iterative solver (All selection,
  Soft sampling, as the paper's Table 1 runs) until it converges or the
  iteration cap; the final partition gives the heterogeneous columns, with
  the improvement 100 (GFLOPS_het / GFLOPS_hom - 1).
"""
from __future__ import annotations

import numpy as np

from . import expand, levels_to_code, make_platform, simulate
from . import solver as V


def metrics(pl, n: int, b: int, levels) -> dict:
    lv = np.ascontiguousarray(levels, np.int8)
    r = simulate(pl, n, b, lv)
    if r["status"] != 0:
        raise ValueError("simulation failed (%d)" % r["status"])
    d = expand(n, b, levels_to_code(n, lv))
    busy = int((r["finish"] - r["start"]).sum())
    T = r["n_tasks"]
    sum_block = int(d["bs"].sum())
    N = n * b
    m = r["makespan"]
    return dict(makespan=m, busy=busy, tasks=T, sum_block=sum_block, depth=1 + int(lv.max()),
                gflops=N ** 3 / 3 / m, load=busy / (pl.n_procs * m), avg_block=sum_block / T)


def table_row(spec, N: int, sizes, order: int, select: int, rp_seed: int, max_level: int, iterations: int,
              seed: int) -> dict:
    pl = make_platform(spec, order=order, select=select, rp_seed=rp_seed)
    homog = []
    for b in sizes:
        n = N // b
        homog.append((b, metrics(pl, n, b, np.zeros(n * (n + 1) * (n + 2) // 6, np.int8))))
    b_best, h = min(homog, key=lambda x: (x[1]["makespan"], -x[0]))
    n = N // b_best
    steps = V.solve(pl, n, b_best, np.zeros(n * (n + 1) * (n + 2) // 6, np.int8), max_level + 1, V.MODE_ALL,
                    V.PICK_SOFT, seed, iterations)
    last = steps[-1]
    final = last.levels
    if last.chosen is not None:  # the cap ended it: apply the last chosen move
        t, dmove = last.chosen >> 1, (-1 if last.chosen & 1 else 1)
        final = last.levels.copy()
        final[t] += dmove
    het = metrics(pl, n, b_best, final)
    return dict(homog=h, homog_block=b_best, het=het, het_levels=np.asarray(final, np.int8),
                improvement=100.0 * (het["gflops"] / h["gflops"] - 1.0), iterations=len(steps))
