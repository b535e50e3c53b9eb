"""Pins of the oracle's performance models and of its FCFS + EFT-P simulation
with write-back caching (HeSP Sec. 2.1), CPU only.

* task and transfer times: hand-derived values, and the defining property of
  a ceiling (rate * (t - 1) < flops <= rate * t) checked with exact fractions
  from flops and rate separately;
* hand-derived schedules (tests/golden/worked_examples.json), including a
  transfer back to host, one message for several blocks from one source, an
  in-flight copy and simultaneous completions;
* one processor: makespan = sum of task times;
* brute force over every (task order, assignment) on tiny DAGs: optimum <=
  oracle, Graham's list-scheduling bound on identical processors, equality on
  chains; an independent replay of the oracle's own choices reproduces every
  start and finish time;
* schedule invariants on random candidates of every workload shape.
"""
import dataclasses
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1602_05510_b300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))
COEF3 = (1, 3, 3, 6)


def plat(key):
    return O.make_platform(W.PLATFORMS[key])


# ------------------------------------------------------------ cost models


def test_exec_ns_hand_values():
    pl = plat("cfg0")
    g = GOLD["exec_ns"]
    assert [O.exec_ns(pl, o, 0, 1024) for o in range(4)] == g["cpu_1024"]
    assert [O.exec_ns(pl, o, 1, 1024) for o in range(4)] == g["gpu_1024"]
    assert [O.exec_ns(pl, o, 0, 512) for o in range(4)] == g["cpu_512"]
    assert [O.exec_ns(pl, o, 1, 512) for o in range(4)] == g["gpu_512"]


def test_xfer_ns_hand_values():
    pl = plat("cfg0")
    g = GOLD["xfer_ns"]
    assert [O.xfer_ns(pl, s * s) for s in g["bs"]] == g["ns"]


@pytest.mark.parametrize("key", ["cfg0", "cfg1b"])
def test_exec_is_ceiling_of_flops_over_rate(key):
    spec = W.PLATFORMS[key]
    pl = O.make_platform(spec)
    for ti, ty in enumerate(spec.types):
        for op in range(4):
            for bs in (1, 2, 3, 7, 64, 128, 256, 300, 512, 1000, 1024, 2048, 4096, 1 << 15):
                flops = Fraction(COEF3[op] * bs ** 3, 3)
                rate = Fraction(ty.peak_gflops * ty.eff_pct[op], 100) * Fraction(bs * bs, bs * bs + ty.h ** 2)
                t = O.exec_ns(pl, op, ti, bs)
                assert rate * (t - 1) < flops <= rate * t


def test_xfer_is_ceiling():
    pl = plat("cfg0")
    for e in (1, 2, 3, 11, 12, 13, 1000, 1 << 20, 3 << 22):
        t = O.xfer_ns(pl, e) - 8000
        assert 12 * (t - 1) < 8 * e <= 12 * t


def test_exec_override():
    spec = dataclasses.replace(W.PLATFORMS["cfg0"], exec_overrides=((3, 1, 512, 12345),))
    pl = O.make_platform(spec)
    assert O.exec_ns(pl, 3, 1, 512) == 12345
    assert O.exec_ns(pl, 3, 1, 1024) == GOLD["exec_ns"]["gpu_1024"][3]


# --------------------------------------------------------- worked examples


@pytest.mark.parametrize("key", ["n2_b1024_all_level0_cpu4_gpu1", "n1_b1024_chol_level1_cpu4_gpu1"])
def test_worked_example_gpu_chain(key):
    e = GOLD[key]
    r = O.simulate(plat(e["platform"]), e["n"], e["b"], e["levels"])
    assert r["status"] == 0
    assert r["makespan"] == e["makespan"]
    assert r["proc"].tolist() == e["proc"]
    assert r["finish"].tolist() == e["finish"]


def test_single_cpu_is_sum_of_task_times():
    pl = O.make_platform(W.single_cpu_platform())
    assert O.simulate(pl, 2, 1024, [0, 0, 0, 0])["makespan"] == GOLD["n2_b1024_single_cpu"]["makespan"]
    rng = np.random.default_rng(1)
    for n in (1, 2, 3, 4):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        d = O.expand(n, 1024, O.levels_to_code(n, lv))
        tot = sum(O.exec_ns(pl, int(o), 0, int(b)) for o, b in zip(d["op"], d["bs"]))
        assert O.simulate(pl, n, 1024, lv)["makespan"] == tot


@pytest.mark.parametrize("key,ncpu", [("n2_b1024_cpu1_gpu1_overrides", 1), ("n3_b1024_cpu2_gpu1_overrides", 2)])
def test_worked_example_with_transfers(key, ncpu):
    e = GOLD[key]
    spec = dataclasses.replace(W.cpu_gpu_platform(ncpu, 1),
                               exec_overrides=tuple(tuple(x) for x in e["overrides"]))
    r = O.simulate(O.make_platform(spec), e["n"], e["b"], e["levels"])
    assert r["status"] == 0
    assert r["makespan"] == e["makespan"]
    assert r["proc"].tolist() == e["proc"]
    assert r["start"].tolist() == e["start"]
    assert r["finish"].tolist() == e["finish"]
    assert r["n_transfers"] == e["n_transfers"]
    assert r["xfer_elems"] == e["xfer_elems"]


# ----------------------------------------------- replay and brute force


def replay(spec, n, b, levels, order, procs, atom_level=None, issue=None, cache=0, links=None):
    """Evaluate a given (task order, assignment) with the caching and
    transfer rules, each task issued at its release time (the latest finish
    of its predecessors), or at issue[j] when given.  cache: 0 write-back,
    1 write-through, 2 write-around.  links: {(src, dst): (latency_ns,
    bytes_per_ns)} for pairs whose cost differs from the platform's.
    Independent of the oracle's event loop."""
    pl = O.make_platform(spec)

    def xfer(s, d, elems):
        if links and (s, d) in links:
            lat, bw = links[(s, d)]
            return lat + -(-(elems * spec.bytes_per_elem) // bw)
        return O.xfer_ns(pl, elems)
    code = O.levels_to_code(n, levels)
    d = O.expand(n, b, code)
    L = int(max(levels)) if atom_level is None else atom_level
    po, pv, _ = O.deps(n, b, code, 1, L)
    a = b >> L
    M = spec.n_mem
    valid = {}
    vfrom = {}

    def atoms(r):
        s = r[2] // a
        return [(r[0] // a + i, r[1] // a + j) for i in range(s) for j in range(s)]

    def is_valid(x, m):
        return valid.get((x, m), m == 0)

    avail = [0] * len(spec.procs)
    start = {}
    fin = {}
    for j, p in zip(order, procs):
        t = max([fin[int(pv[e])] for e in range(po[j], po[j + 1])], default=0)
        if issue is not None:
            assert issue[j] >= t
            t = int(issue[j])
        regs = [tuple(int(v) for v in d["regs"][j][r]) for r in range(int(d["nreg"][j]))]
        m = spec.procs[p][0]
        groups = {}
        xs = []
        drt = 0
        for ri, r in enumerate(regs):
            for x in atoms(r):
                xs.append((x, ri == len(regs) - 1))
                if is_valid(x, m):
                    drt = max(drt, vfrom.get((x, m), 0))
                else:
                    usable = [s for s in range(M) if is_valid(x, s) and vfrom.get((x, s), 0) <= t]
                    if usable:
                        src = min(usable)
                    else:  # only copies still in flight: the one usable first
                        src = min((s for s in range(M) if is_valid(x, s)), key=lambda s: (vfrom.get((x, s), 0), s))
                    groups.setdefault(src, []).append(x)
        arr = {}
        for s, v in groups.items():
            dep = max([t] + [vfrom.get((x, s), 0) for x in v])
            arr[s] = dep + xfer(s, m, len(v) * a * a)
        drt = max([drt] + list(arr.values()))
        ex = O.exec_ns(pl, int(d["op"][j]), spec.procs[p][1], int(d["bs"][j]))
        st = max(t, avail[p], drt)
        for s, v in groups.items():
            for x in v:
                valid[(x, m)] = True
                vfrom[(x, m)] = arr[s]
        written = [x for x, w in xs if w]
        through = st + ex + xfer(m, 0, len(written) * a * a)
        for x in written:
            for mm in range(M):
                valid[(x, mm)] = False
            if cache != 2 or m == 0:
                valid[(x, m)] = True
                vfrom[(x, m)] = st + ex
            if m != 0 and cache != 0:
                valid[(x, 0)] = True
                vfrom[(x, 0)] = through
        avail[p] = st + ex
        start[j], fin[j] = st, st + ex
    return start, fin


REPLAY_CASES = [
    ("cfg0", 3, 1024, None), ("cfg1a", 2, 2048, None), ("cfg1b", 3, 2048, None),
    ("cfg2", 2, 512, None), ("cfg4", 2, 2048, None),
]


@pytest.mark.parametrize("key,n,b,_", REPLAY_CASES)
def test_replay_reproduces_oracle(key, n, b, _):
    rng = np.random.default_rng(hash(key) % 1000)
    spec = W.PLATFORMS[key]
    pl = O.make_platform(spec)
    for _i in range(4):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        r = O.simulate(pl, n, b, lv)
        order = r["order"].tolist()
        s, f = replay(spec, n, b, lv, order, [int(r["proc"][j]) for j in order])
        assert [s[j] for j in range(r["n_tasks"])] == r["start"].tolist()
        assert [f[j] for j in range(r["n_tasks"])] == r["finish"].tolist()


def brute_force_opt(spec, n, b, levels):
    """Smallest makespan over all task orders respecting dependences and all
    assignments, evaluated with `replay` semantics restricted to one memory."""
    pl = O.make_platform(spec)
    code = O.levels_to_code(n, levels)
    d = O.expand(n, b, code)
    po, pv, _ = O.deps(n, b, code, 0)
    T = len(d["op"])
    P = len(spec.procs)
    ex = [[O.exec_ns(pl, int(d["op"][j]), spec.procs[p][1], int(d["bs"][j])) for p in range(P)] for j in range(T)]
    preds = [[int(pv[e]) for e in range(po[j], po[j + 1])] for j in range(T)]
    best = [None]

    def rec(done, fin, avail):
        if len(done) == T:
            ms = max(fin.values())
            if best[0] is None or ms < best[0]:
                best[0] = ms
            return
        for j in range(T):
            if j in done or any(i not in done for i in preds[j]):
                continue
            t = max([fin[i] for i in preds[j]], default=0)
            for p in range(P):
                st = max(t, avail[p])
                if best[0] is not None and st + ex[j][p] >= best[0]:
                    continue
                na = list(avail)
                na[p] = st + ex[j][p]
                fin[j] = na[p]
                rec(done | {j}, fin, na)
                del fin[j]

    rec(frozenset(), {}, [0] * P)
    return best[0]


def identical(P):
    return W.PlatformSpec("id%d" % P, 1, (W.CPU_TYPE,), tuple([(0, 0)] * P))


@pytest.mark.parametrize("n,levels,P", [
    (2, [0, 0, 0, 0], 2), (2, [1, 0, 0, 0], 2), (2, [0, 1, 0, 0], 2), (3, [0] * 10, 2),
    (3, [0] * 10, 3), (2, [0, 0, 1, 0], 3), (1, [1], 2),
])
def test_brute_force_graham(n, levels, P):
    """On identical processors without transfers, FCFS + EFT-P is a greedy
    list schedule: OPT <= makespan <= (2 - 1/P) OPT (Graham 1969)."""
    spec = identical(P)
    r = O.simulate(O.make_platform(spec), n, 1024, levels)
    opt = brute_force_opt(spec, n, 1024, levels)
    assert opt <= r["makespan"]
    assert r["makespan"] * P <= (2 * P - 1) * opt


def test_brute_force_heterogeneous_without_transfers():
    spec = W.big_little_platform()
    spec = dataclasses.replace(spec, procs=((0, 0), (0, 1)))
    for lv in ([0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1]):
        r = O.simulate(O.make_platform(spec), 2, 512, lv)
        assert brute_force_opt(spec, 2, 512, lv) <= r["makespan"]


def test_chain_is_optimal():
    """n = 2 at level 0 is a chain: every schedule runs it in sequence; with
    identical processors the oracle's makespan is the optimum (sum of times)."""
    for P in (1, 2, 3):
        spec = identical(P)
        r = O.simulate(O.make_platform(spec), 2, 1024, [0, 0, 0, 0])
        assert r["makespan"] == brute_force_opt(spec, 2, 1024, [0, 0, 0, 0]) == GOLD["n2_b1024_single_cpu"]["makespan"]


# ------------------------------------------------------------ invariants


def check_invariants(spec, n, b, lv, r):
    pl = O.make_platform(spec)
    code = O.levels_to_code(n, lv)
    d = O.expand(n, b, code)
    po, pv, _ = O.deps(n, b, code, 1, int(max(lv)))
    T = len(d["op"])
    assert r["status"] == 0 and r["n_tasks"] == T
    P = len(spec.procs)
    ex = np.array([O.exec_ns(pl, int(d["op"][j]), spec.procs[int(r["proc"][j])][1], int(d["bs"][j]))
                   for j in range(T)])
    # task time
    assert np.array_equal(r["finish"] - r["start"], ex)
    # precedence
    rel = np.zeros(T, np.int64)
    for j in range(T):
        for e in range(po[j], po[j + 1]):
            assert r["start"][j] >= r["finish"][pv[e]]
            rel[j] = max(rel[j], r["finish"][pv[e]])
    # no processor runs two tasks at once
    for p in range(P):
        idx = np.nonzero(r["proc"] == p)[0]
        s = np.sort(np.stack([r["start"][idx], r["finish"][idx]], 1), axis=0)
        iv = sorted(zip(r["start"][idx].tolist(), r["finish"][idx].tolist()))
        for (a0, a1), (b0, b1) in zip(iv, iv[1:]):
            assert a1 <= b0
    # FCFS: tasks are scheduled in order of (release time, id)
    order = r["order"].tolist()
    keys = [(int(rel[j]), j) for j in order]
    assert keys == sorted(keys)
    # makespan bounds: critical path with the fastest type and no transfers,
    # and total flops over the aggregate peak rate
    ms = r["makespan"]
    assert ms == int(r["finish"].max())
    fastest = [min(O.exec_ns(pl, int(d["op"][j]), ty, int(d["bs"][j])) for ty in range(len(spec.types)))
               for j in range(T)]
    cp = np.zeros(T, np.int64)
    for j in range(T):
        cp[j] = fastest[j] + max([cp[pv[e]] for e in range(po[j], po[j + 1])], default=0)
    assert ms >= cp.max()
    rmax = []
    for (m, ty) in spec.procs:
        tt = spec.types[ty]
        rmax.append(max(Fraction(tt.peak_gflops * tt.eff_pct[int(o)], 100) * Fraction(int(bb) ** 2, int(bb) ** 2 + tt.h ** 2)
                        for o, bb in zip(d["op"], d["bs"])))
    flops = sum(Fraction(COEF3[int(o)] * int(bb) ** 3, 3) for o, bb in zip(d["op"], d["bs"]))
    assert ms * sum(rmax) >= flops
    return d


INV_CASES = [("cfg0", 3, 1024, 2), ("cfg1a", 8, 2048, 3), ("cfg1b", 8, 2048, 3), ("cfg2", 6, 512, 3),
             ("cfg2", 4, 2048, 3), ("cfg4", 5, 2048, 4)]


@pytest.mark.parametrize("key,n,b,nl", INV_CASES)
def test_schedule_invariants(key, n, b, nl):
    rng = np.random.default_rng(n * 31 + b)
    spec = W.PLATFORMS[key]
    pl = O.make_platform(spec)
    for _ in range(3):
        lv = rng.integers(0, nl, O.base_count(n)).astype(np.int8)
        r = O.simulate(pl, n, b, lv)
        check_invariants(spec, n, b, lv, r)


@pytest.mark.parametrize("key,n,b,nl", INV_CASES[:4])
def test_atom_size_and_dependence_mode_do_not_matter(key, n, b, nl):
    rng = np.random.default_rng(5)
    pl = plat(key)
    for _ in range(2):
        lv = rng.integers(0, nl, O.base_count(n)).astype(np.int8)
        L = int(lv.max())
        r1 = O.simulate(pl, n, b, lv, atom_level=L)
        r2 = O.simulate(pl, n, b, lv, atom_level=L + 1)
        for k in ("makespan", "n_transfers", "xfer_elems"):
            assert r1[k] == r2[k]
        for k in ("proc", "start", "finish"):
            assert np.array_equal(r1[k], r2[k])
        if r1["n_tasks"] <= 700:
            r3 = O.simulate(pl, n, b, lv, atom_level=L, dep_mode=0)
            assert np.array_equal(r1["finish"], r3["finish"]) and np.array_equal(r1["proc"], r3["proc"])


def test_gpu_only_fetches_every_touched_element_once():
    """With one GPU and no CPU, host memory is never written again, so every
    element the DAG touches is fetched exactly once."""
    spec = W.PlatformSpec("gpu1", 2, (W.CPU_TYPE, W.GPU_TYPE), ((1, 1),))
    pl = O.make_platform(spec)
    rng = np.random.default_rng(9)
    for n in (1, 2, 3, 5):
        lv = rng.integers(0, 3, O.base_count(n)).astype(np.int8)
        b = 64
        d = O.expand(n, b, O.levels_to_code(n, lv))
        touched = np.zeros((n * b, n * b), bool)
        for j in range(len(d["op"])):
            for r in range(int(d["nreg"][j])):
                r0, c0, s = (int(v) for v in d["regs"][j][r])
                touched[r0:r0 + s, c0:c0 + s] = True
        res = O.simulate(pl, n, b, lv)
        assert res["xfer_elems"] == int(touched.sum())
        assert (res["proc"] == 0).all()


def test_write_invalidates_other_copies():
    """Data written on one side must travel back before the other side reads
    it: in the 1 CPU + 1 GPU worked example the syrk on the CPU waits for the
    block the GPU trsm wrote (start = trsm finish + one block transfer)."""
    e = GOLD["n2_b1024_cpu1_gpu1_overrides"]
    assert e["start"][2] == e["finish"][1] + GOLD["xfer_ns"]["ns"][1]


def test_bad_arguments():
    pl = plat("cfg0")
    assert O.simulate(pl, 2, 1024, [0, 0, 0, -1])["status"] < 0
    assert O.simulate(pl, 2, 1023, [1, 0, 0, 0])["status"] < 0
