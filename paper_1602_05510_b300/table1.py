"""Table 1 of the paper (Sec. 3) on the GPU engine: per scheduling policy,
the best homogeneous partition of a tile-size sweep and the heterogeneous
partition the iterative solver reaches from it, with their GFLOPS, average
load, average block size and DAG depth.

Metrics of one simulated partition of an N x N Cholesky (N = n b):
  GFLOPS = (N^3 / 3) / makespan; load = the tasks' summed execution time /
  (P makespan); avg block = mean block size over the tasks; depth = 1 + the
  deepest split level.
Procedure per platform and policy: simulate the unsplit partition for each
tile size b of the sweep; the smallest makespan (ties to the larger b) is
the homogeneous result; from it, run the iterative solver (All selection,
Soft sampling, as the paper's table) until it converges or hits the
iteration cap; the final partition is the heterogeneous result.

Orchestration only: simulation, metrics and the solver run in libhesp.so.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np

from . import hesp
from . import search as S
from . import workloads as W

POLICIES = (  # (name, order, select), the rows of the paper's table
    ("FCFS/R-P", hesp.ORDER_FCFS, hesp.SELECT_RP), ("PL/R-P", hesp.ORDER_PL, hesp.SELECT_RP),
    ("FCFS/F-P", hesp.ORDER_FCFS, hesp.SELECT_FP), ("PL/F-P", hesp.ORDER_PL, hesp.SELECT_FP),
    ("FCFS/EIT-P", hesp.ORDER_FCFS, hesp.SELECT_EIT), ("PL/EIT-P", hesp.ORDER_PL, hesp.SELECT_EIT),
    ("FCFS/EFT-P", hesp.ORDER_FCFS, hesp.SELECT_EFT), ("PL/EFT-P", hesp.ORDER_PL, hesp.SELECT_EFT),
)


def metrics(plat: "hesp.Platform", n: int, b: int, levels: np.ndarray, max_level: int, task_cap: int = 0) -> Dict:
    """Simulate one partition with its schedule and return its metrics."""
    import torch
    lv = np.ascontiguousarray(levels, np.int8)
    d_lv = torch.from_numpy(lv.copy()).cuda()
    cands = hesp.cands_tensor(n, b, np.zeros(1, np.int64))
    T = hesp.Dag(n, b, max_level).count_tasks(lv)[0]
    cap = max(task_cap, T) if task_cap else 0
    ws = hesp.alloc_workspace(plat, n, max_level, 1, cap)
    sched = (torch.zeros(1, dtype=torch.int64, device="cuda"), torch.empty(T, dtype=torch.int16, device="cuda"),
             torch.empty(T, dtype=torch.int64, device="cuda"), torch.empty(T, dtype=torch.int64, device="cuda"))
    ms, st, _ = hesp.simulate_batch(plat, cands, d_lv, 1, n, max_level, ws, schedule=sched, task_cap=cap)
    busy, nt, sb, dp = hesp.schedule_metrics(cands, d_lv, 1, schedule=sched)
    vals = torch.stack([ms[0], st[0].long(), busy[0], nt[0], sb[0], dp[0].long()]).cpu().numpy()
    m, stt, bz, tasks, sum_block, depth = (int(x) for x in vals)
    if stt != hesp.HESP_OK:
        raise hesp.HespError(stt, "simulation of the partition")
    N = n * b
    return dict(makespan=m, busy=bz, tasks=tasks, sum_block=sum_block, depth=depth, gflops=N ** 3 / 3 / m,
                load=bz / (len(plat.spec.procs) * m), avg_block=sum_block / tasks)


def table_row(spec, N: int, sizes: Sequence[int], order: int, select: int, rp_seed: int, max_level: int,
              iterations: int, seed: int, task_cap: int = 0, ws_bytes=None) -> Dict:
    plat = hesp.Platform(spec, order=order, select=select, rp_seed=rp_seed)
    homog = []
    for b in sizes:
        n = N // b
        homog.append((b, metrics(plat, n, b, np.zeros(W.base_count(n), np.int8), 0)))
    b_best, h = min(homog, key=lambda x: (x[1]["makespan"], -x[0]))
    n = N // b_best
    sv = S.IterativeSolver(spec, n, b_best, max_level + 1, hesp.SOLVER_ALL, hesp.PICK_SOFT, task_cap=task_cap,
                           ws_bytes=ws_bytes, order=order, select=select, rp_seed=rp_seed)
    sv.start(np.zeros(W.base_count(n), np.int8))
    its = 0
    for it in range(iterations):
        chosen, _, _, _ = sv.iterate(seed, it)
        its += 1
        if chosen is None:
            break
    final = sv.cur.cpu().numpy().astype(np.int8)
    het = metrics(plat, n, b_best, final, max_level, task_cap)
    return dict(homog=h, homog_block=b_best, het=het, het_levels=final,
                improvement=100.0 * (het["gflops"] / h["gflops"] - 1.0), iterations=its,
                sweep={b: m["makespan"] for b, m in homog})
