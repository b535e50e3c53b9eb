"""Pins of the iterative-solver oracle (oracle/solver.py, Sec. 2.1
"Iterative solver"), CPU only:

* critical-path flags against a brute-force enumeration of every
  source-to-sink path of small DAGs, and on chains (everything critical);
* Hard takes the best of an independently enumerated set of one-level moves
  (ties to the lower move code) and the makespan falls at every iteration;
* at convergence no one-level move improves the partition;
* Shallow equals All on an unsplit partition, CP is a subset of All and
  equals it when every base task is critical;
* Soft's choice frequencies follow score / sum (statistical), one kept move
  is always taken, and the draw matches SplitMix64 from its published
  definition;
* on cfg0 the converged partition lies between the exhaustive optimum of
  all 1024 partitions and the unsplit partition.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle import solver as V
from paper_1602_05510_b300 import workloads as W


def _dag(n, b, lv):
    code = O.levels_to_code(n, lv)
    d = O.expand(n, b, code)
    po, pv, _ = O.deps(n, b, code, 1, int(max(lv)))
    return d, po, pv


def brute_critical(pl, n, b, lv):
    """Every source-to-sink path, weighted by scheduled durations; flag the
    base tasks of the tasks on a heaviest one."""
    r = O.simulate(pl, n, b, lv)
    d, po, pv = _dag(n, b, lv)
    T = r["n_tasks"]
    dur = (r["finish"] - r["start"]).astype(np.int64)
    succ = [[] for _ in range(T)]
    has_pred = [po[j + 1] > po[j] for j in range(T)]
    for j in range(T):
        for e in range(po[j], po[j + 1]):
            succ[int(pv[e])].append(j)
    paths = []

    def walk(j, acc, path):
        path.append(j)
        acc += int(dur[j])
        if not succ[j]:
            paths.append((acc, list(path)))
        for s in succ[j]:
            walk(s, acc, path)
        path.pop()

    for j in range(T):
        if not has_pred[j]:
            walk(j, 0, [])
    best = max(w for w, _ in paths)
    flags = np.zeros(len(lv), np.int8)
    for w, p in paths:
        if w == best:
            for j in p:
                flags[int(d["base"][j])] = 1
    return flags


@pytest.mark.parametrize("key,n,lv", [
    ("cfg0", 3, [0] * 10), ("cfg0", 3, [1, 0, 0, 0, 0, 0, 0, 0, 0, 0]), ("cfg0", 3, [0, 0, 1, 0, 0, 1, 0, 0, 0, 0]),
    ("cfg0", 2, [1, 1, 0, 1]), ("cfg1b", 3, [0, 1, 0, 0, 0, 0, 0, 1, 0, 0]), ("cfg1a", 2, [2, 0, 0, 1]),
    ("cfg1b", 4, [0] * 20),
])
def test_critical_flags_brute_force(key, n, lv):
    pl = O.make_platform(W.PLATFORMS[key])
    flags, _ = V.critical_bases(pl, n, 1024, lv)
    assert flags.tolist() == brute_critical(pl, n, 1024, lv).tolist()


def test_chain_is_all_critical():
    pl = O.make_platform(W.PLATFORMS["cfg0"])
    for n, lv in ((2, [0, 0, 0, 0]), (1, [2]), (1, [0])):
        flags, _ = V.critical_bases(pl, n, 1024, lv)
        assert flags.tolist() == [1] * len(lv)


def one_level_moves(lv, n_levels, allowed):
    """All moves by one level, enumerated directly: code 2t (split t) when t
    is allowed and not at the deepest level, 2t + 1 (merge t) when t is
    split."""
    out = []
    for t, l in enumerate(lv):
        for d in (+1, -1):
            nl = l + d
            if 0 <= nl < n_levels and (d < 0 or t in allowed):
                w = list(lv)
                w[t] = nl
                out.append((2 * t + (d < 0), w))
    return sorted(out)


@pytest.mark.parametrize("mode", [V.MODE_ALL, V.MODE_CP, V.MODE_SHALLOW])
@pytest.mark.parametrize("key,n,b,NL", [("cfg0", 3, 1024, 2), ("cfg1a", 3, 2048, 3), ("cfg1b", 3, 2048, 3)])
def test_hard_takes_the_best_move(mode, key, n, b, NL):
    pl = O.make_platform(W.PLATFORMS[key])
    rng = np.random.default_rng(mode * 7 + NL)
    lv0 = rng.integers(0, NL, O.base_count(n)).astype(np.int8)
    steps = V.solve(pl, n, b, lv0, NL, mode, V.PICK_HARD, seed=1, iterations=4)
    for s, nxt in zip(steps, steps[1:] + [None]):
        crit, m = V.critical_bases(pl, n, b, s.levels)
        assert m == s.makespan
        allowed = {V.MODE_ALL: set(range(len(s.levels))),
                   V.MODE_CP: {t for t in range(len(s.levels)) if crit[t]},
                   V.MODE_SHALLOW: {t for t in range(len(s.levels)) if s.levels[t] == s.levels.min()}}[mode]
        mv = one_level_moves(s.levels.tolist(), NL, allowed)
        assert [k for k, _ in mv] == s.moves
        ms = [O.simulate(pl, n, b, w, schedule=False)["makespan"] for _, w in mv]
        assert ms == s.makespans
        gain = [s.makespan - x for x in ms]
        if max(gain) <= 0:
            assert s.chosen is None and nxt is None
        else:
            i = gain.index(max(gain))
            assert s.chosen == mv[i][0]
            assert nxt is None or (nxt.makespan == ms[i] and nxt.levels.tolist() == mv[i][1])


@pytest.mark.parametrize("key,n,b,NL", [("cfg0", 3, 1024, 2), ("cfg1b", 3, 2048, 3), ("cfg0", 2, 1024, 3)])
def test_converged_partition_is_a_local_optimum(key, n, b, NL):
    pl = O.make_platform(W.PLATFORMS[key])
    steps = V.solve(pl, n, b, np.zeros(O.base_count(n), np.int8), NL, V.MODE_ALL, V.PICK_HARD, 0, 200)
    last = steps[-1]
    assert last.chosen is None
    assert all(a.makespan > b_.makespan for a, b_ in zip(steps, steps[1:]))
    for _, w in one_level_moves(last.levels.tolist(), NL, set(range(len(last.levels)))):
        assert O.simulate(pl, n, b, w, schedule=False)["makespan"] >= last.makespan


def test_cfg0_converges_between_the_optimum_and_the_start():
    pl = O.make_platform(W.PLATFORMS["cfg0"])
    allv = W.exhaustive_levels(10)
    ms, st, _ = O.simulate_many(pl, 3, 1024, allv)
    assert (st == 0).all()
    for how, seed in ((V.PICK_HARD, 0), (V.PICK_SOFT, 3), (V.PICK_SOFT, 4)):
        steps = V.solve(pl, 3, 1024, np.zeros(10, np.int8), 2, V.MODE_ALL, how, seed, 200)
        assert steps[-1].chosen is None
        assert ms.min() <= steps[-1].makespan <= steps[0].makespan
        assert steps[-1].makespan in set(ms.tolist())


def test_shallow_and_cp_candidate_sets():
    lv0 = np.zeros(10, np.int8)
    a = V.neighbours(lv0, 3, V.MODE_ALL)
    s = V.neighbours(lv0, 3, V.MODE_SHALLOW)
    assert [k for k, _ in a] == [k for k, _ in s]
    lv = np.array([1, 0, 2, 0, 1, 0, 0, 2, 0, 1], np.int8)
    sh = [k for k, _ in V.neighbours(lv, 3, V.MODE_SHALLOW)]
    assert sh == sorted([2 * t for t in range(10) if lv[t] == 0] + [2 * t + 1 for t in range(10) if lv[t] > 0])
    crit = np.array([1, 0, 0, 1, 1, 0, 0, 0, 1, 0], np.int8)
    cp = [k for k, _ in V.neighbours(lv, 3, V.MODE_CP, crit)]
    al = [k for k, _ in V.neighbours(lv, 3, V.MODE_ALL)]
    assert set(cp) <= set(al)
    assert [k for k, _ in V.neighbours(lv, 3, V.MODE_CP, np.ones(10, np.int8))] == al


def test_soft_draw_and_frequencies():
    cur = 1000
    moves = list(range(6))
    ms = [990, 1000, 700, 1200, 940, 999]  # kept scores 10, 300, 60, 1
    kept = {0: 10, 2: 300, 4: 60, 5: 1}
    S = sum(kept.values())
    cnt = dict.fromkeys(kept, 0)
    N = 6000
    for it in range(N):
        i = V.pick(cur, moves, ms, V.PICK_SOFT, seed=42, iteration=it)
        cnt[i] += 1
        # the draw from the generator's published definition (vectorised numpy version)
        u = int(W.counter_u64(42, np.array([it], np.uint64), np.array([0], np.uint64))[0])
        r = (u * S) >> 64
        run = 0
        for j in sorted(kept):
            run += kept[j]
            if run > r:
                assert i == j
                break
    for j, s in kept.items():
        p = s / S
        assert abs(cnt[j] / N - p) <= 4 * np.sqrt(p * (1 - p) / N) + 1e-9, (j, cnt[j])
    # one kept move is always taken; none kept -> None
    for it in range(50):
        assert V.pick(cur, moves, [1000, 1001, 999, 2000, 1000, 1000], V.PICK_SOFT, 5, it) == 2
    assert V.pick(cur, moves, [1000] * 6, V.PICK_SOFT, 5, 0) is None
    assert V.pick(cur, moves, ms, V.PICK_HARD, 0, 0) == 2
    assert V.pick(cur, [0, 1], [900, 900], V.PICK_HARD, 0, 0) == 0


# ------------------------------------------ the solver over partition factors


@pytest.mark.parametrize("mode", [V.MODE_ALL, V.MODE_CP, V.MODE_SHALLOW])
@pytest.mark.parametrize("how", [V.PICK_HARD, V.PICK_SOFT])
def test_factor_solver_with_factors_one_two_is_the_level_solver(mode, how):
    """Factors 1 / 2 are the dyadic levels 0 / 1: with the largest factor 2
    the factor solver makes exactly the level solver's moves (same codes,
    same makespans) from the same start."""
    pl = O.make_platform(W.PLATFORMS["cfg1a"])
    n, b = 3, 2048
    lv0 = np.random.default_rng(mode * 2 + how).integers(0, 2, W.base_count(n)).astype(np.int8)
    a = V.solve(pl, n, b, lv0, 2, mode, how, 99, 8)
    f = V.solve(pl, n, b, lv0 + 1, 2, mode, how, 99, 8, factors=True)
    assert len(a) == len(f)
    for sa, sf in zip(a, f):
        assert np.array_equal(sa.levels + 1, sf.levels)
        assert sa.makespan == sf.makespan and sa.moves == sf.moves and sa.makespans == sf.makespans
        assert sa.chosen == sf.chosen


def test_factor_neighbours_bounds():
    """Values 1 .. 4: a finer move below 4, a coarser move above 1."""
    nb = V.neighbours([1, 2, 4, 3], 4, V.MODE_ALL, factors=True)
    assert [k for k, _ in nb] == [0, 2, 3, 5, 6, 7]
    assert [list(w) for _, w in nb][:2] == [[2, 2, 4, 3], [1, 3, 4, 3]]


def test_factor_solver_improves_and_crit_flags_brute_force():
    """Hard moves lower the makespan at every step on non-dyadic
    partitions, and the factor critical flags equal a brute-force path
    enumeration."""
    pl = O.make_platform(W.PLATFORMS["cfg1a"])
    n, b = 2, 3072
    f0 = np.array([3, 1, 2, 1], np.int8)
    steps = V.solve(pl, n, b, f0, 4, V.MODE_ALL, V.PICK_HARD, 1, 6, factors=True)
    ms = [s.makespan for s in steps]
    assert all(x > y for x, y in zip(ms, ms[1:]))
    # brute force on the factor DAG
    r = O.simulate_factors(pl, n, b, f0)
    code = O.factors_to_code(n, f0)
    d = O.expand(n, b, code)
    po, pv, _ = O.deps_side(n, b, code, b // O.lcm_of(f0))
    T = r["n_tasks"]
    dur = (r["finish"] - r["start"]).astype(np.int64)
    succ = [[] for _ in range(T)]
    for j in range(T):
        for e in range(po[j], po[j + 1]):
            succ[int(pv[e])].append(j)
    best, paths = 0, []

    def walk(j, acc, path):
        path.append(j)
        acc += int(dur[j])
        if not succ[j]:
            paths.append((acc, list(path)))
        for s_ in succ[j]:
            walk(s_, acc, path)
        path.pop()

    for j in range(T):
        if po[j + 1] == po[j]:
            walk(j, 0, [])
    best = max(w for w, _ in paths)
    flags = np.zeros(len(f0), np.int8)
    for w, p in paths:
        if w == best:
            for j in p:
                flags[int(d["base"][j])] = 1
    got, m = V.critical_bases(pl, n, b, f0, factors=True)
    assert m == r["makespan"] and np.array_equal(got, flags)
