"""Pins of the Table 1 metrics oracle (oracle/metrics.py), CPU only:

* one processor: busy time = makespan (load 1);
* busy time = the sum of the per-task model times on the assigned
  processors (exec_ns per task), independent of start and finish;
* uniform level l: average block = b / 2^l exactly, depth = l + 1;
* summed block size = the closed form over base tasks (chol s(s+1)(s+2)/6,
  trsm and syrk s^2(s+1)/2, gemm s^3 tasks of block b / s, s = 2^l);
* GFLOPS x makespan x 3 = N^3;
* the table procedure: the homogeneous block is the best unsplit tile size
  of the sweep, and the solver never makes the heterogeneous partition
  worse (improvement >= 0).
"""
import numpy as np
import pytest

import oracle as O
from oracle import metrics as X
from paper_1602_05510_b300 import workloads as W


def counts(op, l):
    s = 2 ** l
    return [s * (s + 1) * (s + 2) // 6, s * s * (s + 1) // 2, s * s * (s + 1) // 2, s ** 3][op]


@pytest.mark.parametrize("key,n,b", [("cfg0", 3, 1024), ("cfg1a", 4, 2048), ("cfg1b", 4, 2048), ("cfg2", 3, 512)])
def test_metrics_identities(key, n, b):
    spec = W.PLATFORMS[key]
    pl = O.make_platform(spec)
    rng = np.random.default_rng(n)
    for _ in range(3):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        m = X.metrics(pl, n, b, lv)
        r = O.simulate(pl, n, b, lv)
        d = O.expand(n, b, O.levels_to_code(n, lv))
        ex = sum(O.exec_ns(pl, int(d["op"][j]), spec.procs[int(r["proc"][j])][1], int(d["bs"][j]))
                 for j in range(r["n_tasks"]))
        assert m["busy"] == ex
        ops = O.base_ops(n)
        assert m["sum_block"] == sum(counts(int(ops[t]), int(lv[t])) * (b >> int(lv[t])) for t in range(len(lv)))
        assert m["tasks"] == sum(counts(int(ops[t]), int(lv[t])) for t in range(len(lv)))
        assert m["depth"] == 1 + int(lv.max())
        assert abs(m["gflops"] * m["makespan"] * 3 - (n * b) ** 3) <= 1e-6 * (n * b) ** 3
        assert 0 < m["load"] <= 1


def test_single_processor_load_is_one():
    pl = O.make_platform(W.single_cpu_platform())
    for lv in ([0, 0, 0, 0], [1, 0, 2, 1]):
        m = X.metrics(pl, 2, 1024, lv)
        assert m["busy"] == m["makespan"] and m["load"] == 1.0


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_uniform_level_block_and_depth(l):
    pl = O.make_platform(W.PLATFORMS["cfg0"])
    m = X.metrics(pl, 2, 2048, [l] * 4)
    assert m["avg_block"] == 2048 >> l and m["depth"] == l + 1


@pytest.mark.parametrize("order,select", [(0, 0), (1, 3)])
def test_table_row_procedure(order, select):
    spec = W.PLATFORMS["cfg1b"]
    row = X.table_row(spec, 4096, (1024, 2048), order, select, 7, 2, 6, 11)
    pl = O.make_platform(spec, order=order, select=select, rp_seed=7)
    ms = {b: O.simulate(pl, 4096 // b, b, np.zeros(O.base_count(4096 // b), np.int8),
                        schedule=False)["makespan"] for b in (1024, 2048)}
    assert row["homog_block"] == min(ms, key=lambda b: (ms[b], -b))
    assert row["homog"]["makespan"] == ms[row["homog_block"]]
    assert row["het"]["makespan"] <= row["homog"]["makespan"] and row["improvement"] >= 0
    n = 4096 // row["homog_block"]
    assert X.metrics(pl, n, row["homog_block"], row["het_levels"])["makespan"] == row["het"]["makespan"]
