"""Pins of the oracle's other scheduling heuristics of HeSP Sec. 2.1: the
priority-list task order (PL, critical times by backflow of the mean task
time, HEFT-like) and the earliest-idle-time processor choice (EIT-P), CPU only.

* EIT-P equals EFT-P on identical processors sharing one memory (the finish
  order of processors is their idle order there);
* PL equals FCFS on a chain (one order exists);
* PL + EFT-P on identical processors is a list schedule: brute-force OPT <=
  makespan <= (2 - 1/P) OPT;
* PL's order is topological and non-increasing in critical time;
* an independent replay of the oracle's own order and choices reproduces
  every start and finish for all four combinations;
* a hand-derived EIT-P schedule with transfers available.
"""
import dataclasses
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1602_05510_b300 import workloads as W

from test_oracle_sim import brute_force_opt, check_invariants, identical, replay

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


def plat(spec, order, select):
    return O.make_platform(spec, order=order, select=select)


@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_eit_equals_eft_on_identical_processors(P):
    spec = identical(P)
    rng = np.random.default_rng(P)
    for n in (2, 3, 4):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        for order in (O.ORDER_FCFS, O.ORDER_PL):
            a = O.simulate(plat(spec, order, O.SELECT_EFT), n, 1024, lv)
            b = O.simulate(plat(spec, order, O.SELECT_EIT), n, 1024, lv)
            for k in ("proc", "start", "finish"):
                assert np.array_equal(a[k], b[k])


def test_pl_equals_fcfs_on_a_chain():
    for spec in (W.PLATFORMS["cfg0"], W.PLATFORMS["cfg1b"], identical(3)):
        for n, lv in ((2, [0, 0, 0, 0]), (1, [1])):
            for sel in (O.SELECT_EFT, O.SELECT_EIT):
                a = O.simulate(plat(spec, O.ORDER_FCFS, sel), n, 1024, lv)
                b = O.simulate(plat(spec, O.ORDER_PL, sel), n, 1024, lv)
                assert np.array_equal(a["finish"], b["finish"]) and np.array_equal(a["proc"], b["proc"])


@pytest.mark.parametrize("n,levels,P", [(2, [1, 0, 0, 0], 2), (3, [0] * 10, 2), (3, [0] * 10, 3), (2, [0, 1, 0, 0], 3)])
def test_pl_eft_graham_bound(n, levels, P):
    spec = identical(P)
    r = O.simulate(plat(spec, O.ORDER_PL, O.SELECT_EFT), n, 1024, levels)
    opt = brute_force_opt(spec, n, 1024, levels)
    assert opt <= r["makespan"] and r["makespan"] * P <= (2 * P - 1) * opt


def test_pl_order_is_topological_and_by_critical_time():
    spec = W.PLATFORMS["cfg1a"]
    pl = plat(spec, O.ORDER_PL, O.SELECT_EFT)
    rng = np.random.default_rng(3)
    for n in (3, 5):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        r = O.simulate(pl, n, 2048, lv)
        code = O.levels_to_code(n, lv)
        d = O.expand(n, 2048, code)
        po, pv, _ = O.deps(n, 2048, code, 1, int(lv.max()))
        T = len(d["op"])
        pos = np.empty(T, np.int64)
        pos[r["order"]] = np.arange(T)
        for j in range(T):
            for e in range(po[j], po[j + 1]):
                assert pos[pv[e]] < pos[j]
        # critical time: summed task time over processors plus the largest successor's
        w = [sum(O.exec_ns(pl, int(d["op"][j]), ty, int(d["bs"][j])) for (_, ty) in spec.procs) for j in range(T)]
        succ = [[] for _ in range(T)]
        for j in range(T):
            for e in range(po[j], po[j + 1]):
                succ[int(pv[e])].append(j)
        crit = [0] * T
        for j in range(T - 1, -1, -1):
            crit[j] = w[j] + max([crit[s] for s in succ[j]], default=0)
        keys = [(-crit[j], j) for j in r["order"]]
        assert keys == sorted(keys)


@pytest.mark.parametrize("order,select", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("key,n,b", [("cfg0", 3, 1024), ("cfg1a", 3, 2048), ("cfg2", 2, 512), ("cfg1b", 3, 2048)])
def test_replay_and_invariants_all_policies(order, select, key, n, b):
    spec = W.PLATFORMS[key]
    pl = plat(spec, order, select)
    rng = np.random.default_rng(order * 10 + select)
    for _ in range(3):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        r = O.simulate(pl, n, b, lv)
        assert r["status"] == 0
        o = r["order"].tolist()
        s, f = replay(spec, n, b, lv, o, [int(r["proc"][j]) for j in o])
        assert [s[j] for j in range(r["n_tasks"])] == r["start"].tolist()
        assert [f[j] for j in range(r["n_tasks"])] == r["finish"].tolist()
        if order == 0:
            check_invariants(spec, n, b, lv, r)


def test_eit_hand_example_with_transfers_available():
    """1 CPU (p0) + 1 GPU (p1), task times of the golden 'cpu1_gpu1' example:
    under EIT-P both processors are idle whenever a task is released, so the
    lower id (the CPU) takes every task and nothing moves:
    100000 + 10^7 + 200000 + 100000 = 10400000."""
    e = GOLD["n2_b1024_cpu1_gpu1_overrides"]
    spec = dataclasses.replace(W.cpu_gpu_platform(1, 1), exec_overrides=tuple(tuple(x) for x in e["overrides"]))
    r = O.simulate(plat(spec, O.ORDER_FCFS, O.SELECT_EIT), 2, 1024, [0, 0, 0, 0])
    assert r["proc"].tolist() == [0, 0, 0, 0]
    assert r["makespan"] == 10400000 and r["n_transfers"] == 0
