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

F-P and R-P (the processor choice among the processors idle at the task's
release time; a task waits while none is idle):

* on identical processors sharing one memory, F-P equals EIT-P (the idle
  processor with the lowest id is the one that became idle first) and, in
  FCFS order, R-P gives the same start and finish times with other
  processor ids;
* R-P's choice on a chain (every processor idle) is the SplitMix64 draw of
  the task id, computed here from the generator's published definition;
* F-P on the cfg0 chain is the EFT-P worked example (the GPU is idle and
  fastest every time); at a fork on one big and one LITTLE core F-P puts the
  second task on the idle LITTLE core where EFT-P would queue it on big;
* a definition check on shared-memory platforms: every task starts at or
  after its release, waits only while every processor is busy, is served in
  first-come first-served order (release time, then id), and takes the
  fastest (F-P) or the drawn (R-P) processor among those idle for it;
* with transfers: a replay at the oracle's issue times reproduces every
  start and finish, and the chosen processor was idle at the issue time.
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


# ---------------------------------------------------------------- F-P, R-P

def rp_pick(seed, j, m):
    """R-P's draw for task j among m idle processors: SplitMix64 counter
    value u(seed, c = j, k = 0), then Lemire's multiply-shift into [0, m)."""
    u = W.counter_u64(seed, np.array([j], np.uint64), np.array([0], np.uint64))
    return int(W.draw(u, m)[0])


@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_fp_rp_on_identical_processors(P):
    spec = identical(P)
    rng = np.random.default_rng(40 + P)
    for n in (2, 3, 4):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        for order in (O.ORDER_FCFS, O.ORDER_PL):
            e = O.simulate(plat(spec, order, O.SELECT_EIT), n, 1024, lv)
            f = O.simulate(plat(spec, order, O.SELECT_FP), n, 1024, lv)
            r = O.simulate(O.make_platform(spec, order=order, select=O.SELECT_RP, rp_seed=99), n, 1024, lv)
            assert e["status"] == f["status"] == r["status"] == 0
            for k in ("proc", "start", "finish"):
                assert np.array_equal(e[k], f[k])
            if order == O.ORDER_FCFS:
                # time only moves forward, so every processor idle at t is as
                # good as another; under PL a later task may be released
                # earlier, and then which idle processor was taken matters
                assert np.array_equal(e["start"], r["start"]) and np.array_equal(e["finish"], r["finish"])


@pytest.mark.parametrize("P,seed", [(2, 0), (3, 7), (5, 123456789), (13, 2 ** 63 + 5)])
def test_rp_draws_on_a_chain(P, seed):
    for n, lv in ((2, [0, 0, 0, 0]), (1, [1]), (1, [2])):
        for order in (O.ORDER_FCFS, O.ORDER_PL):
            r = O.simulate(O.make_platform(identical(P), order=order, select=O.SELECT_RP, rp_seed=seed), n, 1024, lv)
            assert r["status"] == 0
            if n == 1 and lv == [2]:
                continue  # not a chain (the level-1 trsm has parallel halves)
            want = [rp_pick(seed, j, P) for j in range(r["n_tasks"])]
            assert r["proc"].tolist() == want


def test_fp_chain_is_the_eft_worked_example():
    g = GOLD["n2_b1024_all_level0_cpu4_gpu1"]
    for order in (O.ORDER_FCFS, O.ORDER_PL):
        r = O.simulate(plat(W.PLATFORMS["cfg0"], order, O.SELECT_FP), 2, 1024, [0, 0, 0, 0])
        assert r["proc"].tolist() == [4, 4, 4, 4]
        assert r["finish"].tolist() == g["finish"] and r["makespan"] == g["makespan"]


def test_fp_fork_takes_the_idle_slow_core():
    """n = 3, base tasks chol(0), trsm(0,1), trsm(0,2), ... on one big (p0)
    and one LITTLE (p1) core sharing memory: both trsm are released when the
    chol ends; F-P gives the first to big and the second to the idle LITTLE
    core, EFT-P queues the second on big (four times faster)."""
    spec = W.PlatformSpec("big1_little1", 1, (W.BIG_TYPE, W.LITTLE_TYPE), ((0, 0), (0, 1)))
    f = O.simulate(plat(spec, O.ORDER_FCFS, O.SELECT_FP), 3, 1024, [0] * 10)
    e = O.simulate(plat(spec, O.ORDER_FCFS, O.SELECT_EFT), 3, 1024, [0] * 10)
    c0 = int(f["finish"][0])
    assert f["proc"][:3].tolist() == [0, 0, 1] and f["start"][1] == f["start"][2] == c0
    assert e["proc"][:3].tolist() == [0, 0, 0] and e["start"][2] == e["finish"][1]
    pl = O.make_platform(spec)
    assert f["finish"][2] - c0 == O.exec_ns(pl, O.OP_TRSM, 1, 1024)


def _dag(n, b, lv):
    code = O.levels_to_code(n, lv)
    d = O.expand(n, b, code)
    po, pv, _ = O.deps(n, b, code, 1, int(max(lv)))
    return d, po, pv


def check_fcfs_idle_choice(spec, n, b, lv, r, select, seed):
    """The FCFS rules for F-P / R-P on one shared memory, from their
    definition: release r_j = latest predecessor finish; a task starts at or
    after its release, waits only while every processor is busy, is served
    in (release, id) order, and takes the fastest (F-P, ties to the lower
    id) or the drawn (R-P) processor among those idle for it."""
    pl = O.make_platform(spec)
    d, po, pv = _dag(n, b, lv)
    T = r["n_tasks"]
    P = len(spec.procs)
    proc, st, fi = r["proc"].astype(int), r["start"].astype(np.int64), r["finish"].astype(np.int64)
    assert np.array_equal(r["issue"], st)  # one memory: no data to wait for
    rel = np.array([max([fi[pv[e]] for e in range(po[j], po[j + 1])], default=0) for j in range(T)], np.int64)
    fifo = sorted(range(T), key=lambda j: (rel[j], j))
    rank = np.empty(T, np.int64)
    rank[fifo] = np.arange(T)
    on = [[k for k in range(T) if proc[k] == p] for p in range(P)]

    def busy(p, tau):
        return any(st[k] <= tau < fi[k] for k in on[p])

    for j in range(T):
        assert st[j] >= rel[j]
        if st[j] > rel[j]:
            instants = {int(rel[j])} | {int(f) for f in fi if rel[j] < f < st[j]}
            for tau in instants:
                assert all(busy(p, tau) for p in range(P)), (j, tau)
        # idle for j at st[j]: nothing running there, and not taken at that
        # instant by a task ahead of j in the queue
        idle = [p for p in range(P)
                if all(fi[k] <= st[j] or st[k] > st[j] or (st[k] == st[j] and rank[k] > rank[j])
                       for k in on[p] if k != j)]
        assert proc[j] in idle
        if select == O.SELECT_FP:
            ex = {p: O.exec_ns(pl, int(d["op"][j]), spec.procs[p][1], int(d["bs"][j])) for p in idle}
            assert proc[j] == min(idle, key=lambda p: (ex[p], p))
        else:
            assert proc[j] == idle[rp_pick(seed, j, len(idle))]
    # first-come first-served: a task queued earlier never starts later
    for a, b_ in zip(fifo, fifo[1:]):
        assert st[a] <= st[b_]


@pytest.mark.parametrize("select", [2, 3])
@pytest.mark.parametrize("spec_key,n", [("cfg1b", 3), ("cfg1b", 4), ("id3", 4), ("bl11", 3)])
def test_fcfs_fp_rp_definition(select, spec_key, n):
    spec = {"cfg1b": W.PLATFORMS["cfg1b"], "id3": identical(3),
            "bl11": W.PlatformSpec("big1_little1", 1, (W.BIG_TYPE, W.LITTLE_TYPE), ((0, 0), (0, 1)))}[spec_key]
    rng = np.random.default_rng(select * 100 + n)
    for rep_ in range(3):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        seed = 1000 + rep_
        r = O.simulate(O.make_platform(spec, order=O.ORDER_FCFS, select=select, rp_seed=seed), n, 2048, lv)
        assert r["status"] == 0
        check_fcfs_idle_choice(spec, n, 2048, lv, r, select, seed)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("select", [2, 3])
@pytest.mark.parametrize("key,n,b", [("cfg0", 3, 1024), ("cfg1a", 3, 2048), ("cfg2", 2, 512), ("cfg2", 3, 1024)])
def test_fp_rp_replay_with_transfers(order, select, key, n, b):
    """Replay at the oracle's issue times reproduces every start and finish;
    the chosen processor was idle at the issue time (its previous task
    finished by then); under PL a task is issued at its release time when a
    processor is idle then, else when the first one becomes idle; under
    FCFS no task is issued before its release and the issue order follows
    (release, id)."""
    spec = W.PLATFORMS[key]
    rng = np.random.default_rng(order * 10 + select + n)
    for rep_ in range(3):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        seed = 77 + rep_
        pl = O.make_platform(spec, order=order, select=select, rp_seed=seed)
        r = O.simulate(pl, n, b, lv)
        assert r["status"] == 0
        o = r["order"].tolist()
        s_, f_ = replay(spec, n, b, lv, o, [int(r["proc"][j]) for j in o], issue=r["issue"])
        assert [s_[j] for j in range(r["n_tasks"])] == r["start"].tolist()
        assert [f_[j] for j in range(r["n_tasks"])] == r["finish"].tolist()
        d, po, pv = _dag(n, b, lv)
        fi = r["finish"]
        avail = [0] * len(spec.procs)
        rel_seen = []
        for j in o:
            rel = max([int(fi[pv[e]]) for e in range(po[j], po[j + 1])], default=0)
            t = int(r["issue"][j])
            p = int(r["proc"][j])
            idle = [q for q in range(len(spec.procs)) if avail[q] <= t]
            assert p in idle
            if order == O.ORDER_PL:
                assert t == (rel if any(a <= rel for a in avail) else min(avail))
            else:
                assert t >= rel
                rel_seen.append((rel, j, t))
            if select == O.SELECT_FP:
                ex = {q: O.exec_ns(pl, int(d["op"][j]), spec.procs[q][1], int(d["bs"][j])) for q in idle}
                assert p == min(idle, key=lambda q: (ex[q], q))
            else:
                assert p == idle[rp_pick(seed, j, len(idle))]
            avail[p] = int(fi[j])
        if order == O.ORDER_FCFS:
            by_queue = sorted(rel_seen)
            assert [x[2] for x in by_queue] == sorted(x[2] for x in by_queue)


# ---------------------------------------------------------------- WT, WA

def test_write_around_worked_example():
    g = GOLD["n2_b1024_cpu4_gpu1_write_around"]
    r = O.simulate(O.make_platform(W.PLATFORMS["cfg0"], cache=O.CACHE_WA), 2, 1024, g["levels"])
    assert r["proc"].tolist() == g["proc"] and r["start"].tolist() == g["start"]
    assert r["finish"].tolist() == g["finish"] and r["makespan"] == g["makespan"]
    wt = O.simulate(O.make_platform(W.PLATFORMS["cfg0"], cache=O.CACHE_WT), 2, 1024, g["levels"])
    assert wt["makespan"] == g["write_through_makespan"] == GOLD["n2_b1024_all_level0_cpu4_gpu1"]["makespan"]


def test_write_through_and_around_on_the_transfer_back_example():
    e = GOLD["n2_b1024_cpu1_gpu1_overrides"]
    spec = dataclasses.replace(W.cpu_gpu_platform(1, 1), exec_overrides=tuple(tuple(x) for x in e["overrides"]))
    for cache in (O.CACHE_WT, O.CACHE_WA):
        r = O.simulate(O.make_platform(spec, cache=cache), 2, 1024, [0, 0, 0, 0])
        assert r["proc"].tolist() == e["proc"] and r["finish"].tolist() == e["finish"]
        assert r["n_transfers"] == 1


@pytest.mark.parametrize("key", ["cfg1b", "id3"])
def test_caches_coincide_with_one_memory(key):
    spec = W.PLATFORMS["cfg1b"] if key == "cfg1b" else identical(3)
    rng = np.random.default_rng(8)
    for n in (3, 4):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        rs = [O.simulate(O.make_platform(spec, cache=c), n, 1024, lv) for c in (0, 1, 2)]
        for r in rs[1:]:
            assert np.array_equal(r["start"], rs[0]["start"]) and np.array_equal(r["proc"], rs[0]["proc"])


@pytest.mark.parametrize("cache", [1, 2])
@pytest.mark.parametrize("order,select", [(0, 0), (1, 1), (0, 2)])
@pytest.mark.parametrize("key,n,b", [("cfg0", 3, 1024), ("cfg1a", 3, 2048), ("cfg2", 3, 512), ("cfg4", 2, 2048)])
def test_cache_replay(cache, order, select, key, n, b):
    """An independent replay of the oracle's order, choices and issue times
    under WT / WA reproduces every start and finish."""
    spec = W.PLATFORMS[key]
    rng = np.random.default_rng(cache * 100 + order * 10 + select + n)
    for rep_ in range(3):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        r = O.simulate(O.make_platform(spec, order=order, select=select, rp_seed=5, cache=cache), n, b, lv)
        assert r["status"] == 0
        o = r["order"].tolist()
        s_, f_ = replay(spec, n, b, lv, o, [int(r["proc"][j]) for j in o], issue=r["issue"], cache=cache)
        assert [s_[j] for j in range(r["n_tasks"])] == r["start"].tolist()
        assert [f_[j] for j in range(r["n_tasks"])] == r["finish"].tolist()


# ---------------------------------------------------------------- network topology

def test_link_costs_worked_example():
    g = GOLD["n2_b1024_cpu4_gpu1_fast_host_link"]
    links = {(s, d): (lat, bw) for s, d, lat, bw in g["links"]}
    r = O.simulate(O.make_platform(W.PLATFORMS["cfg0"], links=links), 2, 1024, g["levels"])
    assert r["proc"].tolist() == g["proc"] and r["finish"].tolist() == g["finish"]
    r2 = O.simulate(O.make_platform(W.PLATFORMS["cfg0"], links={(1, 0): (1000, 24)}), 2, 1024, g["levels"])
    assert r2["makespan"] == GOLD["n2_b1024_all_level0_cpu4_gpu1"]["makespan"]


def test_uniform_links_equal_the_scalar_model():
    spec = W.PLATFORMS["cfg2"]
    uni = {(s, d): (spec.xfer_latency_ns, spec.bw_bytes_per_ns) for s in range(3) for d in range(3) if s != d}
    rng = np.random.default_rng(21)
    for _ in range(3):
        lv = rng.integers(0, 3, O.base_count(3)).astype(np.int8)
        a = O.simulate(O.make_platform(spec), 3, 1024, lv)
        b = O.simulate(O.make_platform(spec, links=uni), 3, 1024, lv)
        assert np.array_equal(a["start"], b["start"]) and np.array_equal(a["proc"], b["proc"])


@pytest.mark.parametrize("cache", [0, 1, 2])
@pytest.mark.parametrize("key,n,b", [("cfg2", 3, 1024), ("cfg4", 2, 2048), ("cfg1a", 3, 2048)])
def test_link_replay(cache, key, n, b):
    """Asymmetric per-link costs (a fast GPU-GPU link, slow host links): an
    independent replay reproduces every start and finish."""
    spec = W.PLATFORMS[key]
    links = {(0, 1): (20000, 6), (1, 0): (15000, 9)}
    if spec.n_mem > 2:
        links.update({(1, 2): (1000, 50), (2, 1): (1500, 40), (0, 2): (9000, 12), (2, 0): (4000, 30)})
    rng = np.random.default_rng(cache + n)
    for _ in range(3):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        r = O.simulate(O.make_platform(spec, cache=cache, links=links), n, b, lv)
        assert r["status"] == 0
        o = r["order"].tolist()
        s_, f_ = replay(spec, n, b, lv, o, [int(r["proc"][j]) for j in o], cache=cache, links=links)
        assert [s_[j] for j in range(r["n_tasks"])] == r["start"].tolist()
        assert [f_[j] for j in range(r["n_tasks"])] == r["finish"].tolist()


# ---- PL pinned by a schedule worked out by hand (golden file), where PL
# and FCFS differ, and two mistakes planted in a copy of the oracle's C source
# (own time counted once per processor type; ties to the higher id), each of
# which the pin catches.

PLX = GOLD["n2_b1024_syrk_split_pl_vs_fcfs_p3"]


def plx_spec():
    return dataclasses.replace(W.big_little_platform(), procs=tuple(tuple(p) for p in PLX["procs"]),
                               exec_overrides=tuple(tuple(x) for x in PLX["overrides"]))


def plx_run(order):
    return O.simulate(plat(plx_spec(), order, O.SELECT_EFT), PLX["n"], PLX["b"], PLX["levels"])


def plx_matches(r, want):
    return (r["status"] == 0 and r["makespan"] == want["makespan"] and r["proc"].tolist() == want["proc"]
            and r["start"].tolist() == want["start"] and r["finish"].tolist() == want["finish"])


def test_pl_hand_derived_schedule():
    r = plx_run(O.ORDER_PL)
    assert plx_matches(r, PLX["pl"]), (r["proc"], r["start"], r["finish"])
    assert r["order"].tolist() == PLX["pl_order"]
    f = plx_run(O.ORDER_FCFS)
    assert plx_matches(f, PLX["fcfs"]), (f["proc"], f["start"], f["finish"])
    assert r["proc"].tolist() != f["proc"].tolist()  # the two orders give different schedules
    # the DAG of the example: predecessors as listed in the golden file
    code = O.levels_to_code(PLX["n"], PLX["levels"])
    po, pv, _ = O.deps(PLX["n"], PLX["b"], code, 1, 1)
    assert [sorted(pv[po[j]:po[j + 1]].tolist()) for j in range(len(po) - 1)] == PLX["predecessors"]


def _plant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(O.__file__), "hesp_oracle.c")).read()
    assert src.count(old) == 1, name
    return O.build_variant(src.replace(old, new), str(tmp_path / ("lib_%s.so" % name)))


PL_PLANTS = {
    # own time summed over processor types instead of processors
    "per_type": ("for (int p = 0; p < P; p++) w += or_exec_ns(pl, d.t[j].op, pl->proc_type[p], d.t[j].bs);",
                 "for (int p = 0; p < pl->n_types; p++) w += or_exec_ns(pl, d.t[j].op, p, d.t[j].bs);"),
    # equal critical times ordered by decreasing id
    "tie_high": ("    return i < j ? -1 : (i > j);\n}", "    return i > j ? -1 : (i < j);\n}"),
}


@pytest.mark.parametrize("name", sorted(PL_PLANTS))
def test_pl_pin_catches_planted_mistake(tmp_path, name):
    path = _plant(tmp_path, name, *PL_PLANTS[name])
    with O.using_library(path):
        r = plx_run(O.ORDER_PL)
        f = plx_run(O.ORDER_FCFS)
    assert not plx_matches(r, PLX["pl"])
    assert plx_matches(f, PLX["fcfs"])  # the planted mistakes touch PL only
    assert plx_matches(plx_run(O.ORDER_PL), PLX["pl"])  # the real oracle again
