"""Pins of the oracle's general partition parameter (CPU only).

Sec. 2.1 "Iterative solver": a partition cuts a task's data blocks of size d
into blocks of size p d, p in (0, 1].  The oracle's one-level k-way
partitions take p = 1 / k per base task (factor k); k = 2 is the 2x2
partition of Fig. 3 and k = 3 next to k = 2 gives the non-dyadic tilings of
Fig. 4, whose partially overlapping blocks the atoms (side b / lcm of the
factors) intersect.  These tests pin it to facts fixed independently of its
code:

* task counts per op against closed forms (tetrahedral, k^2 (k+1) / 2, k^3);
* a chol cut k ways is exactly the Fig. 1 loop on k tiles of size b / k
  (same tasks, same order, same simulated schedule);
* factors 1 / 2 give exactly the dyadic levels 0 / 1;
* the flop total N^3 / 3 for every factor vector;
* running the tasks as real linear algebra gives numpy's Cholesky factor,
  in creation order and in random orders allowed by the derived dependences;
* all-pairs dependences and the atom version agree on non-dyadic mixes, WaR
  never fires, and halving the atom side changes nothing;
* the hand-derived dependences of the intersecting blocks of Fig. 4;
* on one processor the makespan is the sum of the task times.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_05510_b300 import workloads as W

from test_oracle_dag import _run_numeric, _upper_blocks_close, closure_pairs


def fcode(n, factors):
    return O.factors_to_code(n, np.asarray(factors, np.int8))


def closed_count(op, k):
    if op == O.OP_CHOL:
        return k * (k + 1) * (k + 2) // 6
    if op == O.OP_GEMM:
        return k ** 3
    return k * k * (k + 1) // 2


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_counts_closed_form(k):
    n = 3  # base ops chol, trsm, trsm, gemm, syrk, syrk, ...: every op occurs
    ops = O.base_ops(n)
    for t, op in enumerate(ops):
        f = np.ones(len(ops), np.int8)
        f[t] = k
        d = O.expand(n, 60, fcode(n, f))
        assert len(d["op"]) == len(ops) - 1 + closed_count(int(op), k)
        assert int((d["base"] == t).sum()) == closed_count(int(op), k)
        assert set(d["bs"][d["base"] == t].tolist()) == {60 // k}


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_chol_factor_k_is_fig1_on_k_tiles(k):
    b = 60
    d1 = O.expand(1, b, fcode(1, [k]))
    dk = O.expand(k, b // k, O.levels_to_code(k, np.zeros(O.base_count(k), np.int8)))
    assert np.array_equal(d1["op"], dk["op"])
    assert np.array_equal(d1["regs"], dk["regs"])
    spec = W.PLATFORMS["cfg0"]
    pl = O.make_platform(spec)
    r1 = O.simulate_factors(pl, 1, 3840, [k])
    rk = O.simulate(pl, k, 3840 // k, np.zeros(O.base_count(k), np.int8))
    assert r1["status"] == 0 and rk["status"] == 0
    for key in ("makespan", "n_tasks", "xfer_elems", "n_transfers"):
        assert r1[key] == rk[key], key
    for key in ("proc", "start", "finish", "order"):
        assert np.array_equal(r1[key], rk[key]), key


@pytest.mark.parametrize("seed", range(6))
def test_factors_one_two_are_levels_zero_one(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 6))
    lv = rng.integers(0, 2, O.base_count(n)).astype(np.int8)
    assert np.array_equal(fcode(n, lv + 1), O.levels_to_code(n, lv))
    for key in ("cfg0", "cfg1a"):
        pl = O.make_platform(W.PLATFORMS[key])
        a = O.simulate_factors(pl, n, 2048, lv + 1)
        b = O.simulate(pl, n, 2048, lv)
        assert a["status"] == 0 and a["makespan"] == b["makespan"]
        assert np.array_equal(a["proc"], b["proc"]) and np.array_equal(a["finish"], b["finish"])


def test_flops_sum_is_n_cubed_over_3():
    rng = np.random.default_rng(5)
    coef = np.array([1, 3, 3, 6], np.int64)
    for n in (1, 2, 3, 5):
        for _ in range(6):
            f = rng.integers(1, 5, O.base_count(n)).astype(np.int8)
            d = O.expand(n, 1200, fcode(n, f))
            assert int((coef[d["op"]] * d["bs"] ** 3).sum()) == (n * 1200) ** 3


@pytest.mark.parametrize("seed", range(8))
def test_numeric_execution_gives_cholesky(seed):
    """The k-way blocked algorithms, run as real linear algebra (upper
    storage, A = U^T U), give numpy's Cholesky factor in creation order and
    in random orders that respect the atom dependences (atoms of side
    b / lcm of the factors)."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 4))
    b = 12
    f = rng.integers(1, 5, O.base_count(n)).astype(np.int8)
    N = n * b
    G = rng.standard_normal((N, N))
    A = G @ G.T + N * np.eye(N)
    U = np.linalg.cholesky(A).T
    code = fcode(n, f)
    d = O.expand(n, b, code)
    T = len(d["op"])
    assert _upper_blocks_close(_run_numeric(n, b, d, range(T), A), U, n, b)
    po, pv, war = O.deps_side(n, b, code, b // O.lcm_of(f))
    assert war == 0
    for _ in range(3):
        pend = np.diff(po).copy()
        succ = [[] for _ in range(T)]
        for j in range(T):
            for e in range(po[j], po[j + 1]):
                succ[int(pv[e])].append(j)
        ready = [j for j in range(T) if pend[j] == 0]
        order = []
        while ready:
            j = ready.pop(int(rng.integers(len(ready))))
            order.append(j)
            for s in succ[j]:
                pend[s] -= 1
                if pend[s] == 0:
                    ready.append(s)
        assert len(order) == T
        assert _upper_blocks_close(_run_numeric(n, b, d, order, A), U, n, b)


@pytest.mark.parametrize("seed", range(8))
def test_allpairs_equals_atoms_non_dyadic(seed):
    rng = np.random.default_rng(40 + seed)
    n = int(rng.integers(1, 4))
    f = rng.choice(np.array([1, 2, 3, 4], np.int8), O.base_count(n))
    f[0] = 3  # at least one non-dyadic factor
    b = 24
    code = fcode(n, f)
    a = O.deps(n, b, code, 0)
    side = b // O.lcm_of(f)
    c1 = O.deps_side(n, b, code, side)
    c2 = O.deps_side(n, b, code, side // 2)
    assert c1[2] == 0 and c2[2] == 0
    assert closure_pairs(c1[0], c1[1]) == closure_pairs(a[0], a[1])
    assert np.array_equal(c1[0], c2[0]) and np.array_equal(c1[1], c2[1])
    with pytest.raises(ValueError):  # atoms coarser than the common refinement
        O.deps_side(n, b, code, side * 5)


def test_fig4_intersecting_blocks():
    """Fig. 4: the tile Q2 = A01 of a 2 x 2 tiled matrix is tiled two ways,
    2 x 2 by the trsm that writes it (factor 2) and 3 x 3 by the syrk that
    reads it (factor 3).  Derived by hand on b = 6 (trsm blocks 3 x 3, syrk
    blocks 2 x 2): the trsm tasks writing A01's blocks are, in creation
    order, ids 1 (rows 0:3, cols 0:3), 2 (0:3, 3:6), 5 (3:6, 0:3) and
    6 (3:6, 3:6).  The syrk block A01[p][i] (rows 2p:2p+2, cols 2i:2i+2)
    then depends on every one of them it meets: [0][0] only on 1, [0][1] on
    1 and 2, [1][1] on all four, [2][2] only on 6."""
    n, b = 2, 6
    f = np.array([1, 2, 3, 1], np.int8)  # chol(0), trsm(0,1), syrk(0,1), chol(1)
    code = fcode(n, f)
    d = O.expand(n, b, code)
    trsm_writes = {j: tuple(d["regs"][j][1]) for j in range(len(d["op"])) if d["base"][j] == 1}
    writers = {j: r for j, r in trsm_writes.items() if d["op"][j] in (O.OP_TRSM, O.OP_GEMM)}
    assert {j: r for j, r in writers.items() if d["op"][j] == O.OP_TRSM} == {
        1: (0, 6, 3), 2: (0, 9, 3), 5: (3, 6, 3), 6: (3, 9, 3)}
    po, pv, war = O.deps_side(n, b, code, 1)
    assert war == 0

    def preds(j):
        return set(int(x) for x in pv[po[j]:po[j + 1]])

    # the syrk tasks of the factor-3 syrk: syrk(A01[p][i] -> C_ii) reads one block of A01
    syrk_tasks = [j for j in range(len(d["op"])) if d["base"][j] == 2 and d["op"][j] == O.OP_SYRK]
    readers = {}
    for j in syrk_tasks:
        r0 = tuple(int(v) for v in d["regs"][j][0])  # block of A01 read first
        readers.setdefault(r0, j)
    first = lambda p, i: readers[(2 * p, 6 + 2 * i, 2)]
    trsm_ids = {1, 2, 5, 6}
    assert preds(first(0, 0)) & trsm_ids == {1}
    assert preds(first(0, 1)) & trsm_ids == {1, 2}
    assert preds(first(1, 1)) & trsm_ids == {1, 2, 5, 6}
    assert preds(first(2, 2)) & trsm_ids == {6}


@pytest.mark.parametrize("seed", range(4))
def test_one_processor_makespan_is_sum_of_task_times(seed):
    rng = np.random.default_rng(70 + seed)
    n = int(rng.integers(1, 5))
    f = rng.integers(1, 5, O.base_count(n)).astype(np.int8)
    spec = {"n_mem": 1, "types": [{"peak_gflops": 30, "h": 256, "eff_pct": [70, 80, 85, 90]}],
            "procs": [(0, 0)], "xfer_latency_ns": 0, "bytes_per_elem": 8, "bw_bytes_per_ns": 1}
    pl = O.make_platform(spec)
    b = 3072
    r = O.simulate_factors(pl, n, b, f)
    d = O.expand(n, b, fcode(n, f))
    want = sum(O.exec_ns(pl, int(op), 0, int(bs)) for op, bs in zip(d["op"], d["bs"]))
    assert r["status"] == 0 and r["makespan"] == want


def test_bad_factor_vectors():
    pl = O.make_platform(W.PLATFORMS["cfg0"])
    assert O.simulate_factors(pl, 2, 2048, [3, 1, 1, 1])["status"] != 0  # 3 does not divide 2048
    assert O.simulate_factors(pl, 2, 2048, [0, 1, 1, 1])["status"] != 0
    assert O.simulate_factors(pl, 2, 3072, [3, 1, 2, 4])["status"] == 0  # 12 divides 3072
