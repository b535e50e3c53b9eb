"""GPU iterative partition solver (hesp_simulate_critical, hesp_solver_moves,
hesp_solver_pick) against the oracle (oracle/solver.py): critical-path flags
per base task bit-exact, and whole solver trajectories -- partition and
makespan at each iteration, the candidate moves, their simulated makespans
and the chosen move -- identical for every selection policy and sampling
type."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import solver as V  # noqa: E402
from paper_1602_05510_b300 import hesp  # noqa: E402
from paper_1602_05510_b300 import search as S  # noqa: E402
from paper_1602_05510_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


@pytest.mark.parametrize("order,select", [(0, 0), (1, 0), (0, 2)])
@pytest.mark.parametrize("key,n,b,NL,C", [("cfg0", 3, 1024, 2, 64), ("cfg1a", 8, 2048, 3, 24),
                                          ("cfg1b", 8, 2048, 3, 24), ("cfg2", 6, 512, 3, 24),
                                          ("cfg4", 5, 2048, 4, 12)])
def test_critical_flags_parity(order, select, key, n, b, NL, C):
    spec = W.PLATFORMS[key]
    nb = W.base_count(n)
    lv = np.random.default_rng(n * 10 + NL + order).integers(0, NL, (C, nb)).astype(np.int8)
    plat = hesp.Platform(spec, order=order, select=select, rp_seed=5)
    d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * nb)
    ws = hesp.alloc_workspace(plat, n, NL - 1, C)
    crit = torch.full((C * nb,), -1, dtype=torch.int8, device="cuda")
    ms, st = hesp.simulate_critical(plat, cands, d_lv, C, n, NL - 1, ws, crit)
    torch.cuda.synchronize()
    ms, st, crit = ms.cpu().numpy(), st.cpu().numpy(), crit.cpu().numpy().reshape(C, nb)
    pl = O.make_platform(spec, order=order, select=select, rp_seed=5)
    for c in range(C):
        f, m = V.critical_bases(pl, n, b, lv[c])
        assert st[c] == 0 and ms[c] == m, c
        assert np.array_equal(crit[c], f), c
        assert crit[c].any()


def same_trajectory(g, o):
    assert len(g) == len(o)
    for a, e in zip(g, o):
        assert a.levels.tolist() == e.levels.tolist()
        assert a.makespan == e.makespan
        assert a.moves == e.moves
        assert a.makespans == e.makespans
        assert a.chosen == e.chosen


@pytest.mark.parametrize("mode", [hesp.SOLVER_ALL, hesp.SOLVER_CP, hesp.SOLVER_SHALLOW])
@pytest.mark.parametrize("pick", [hesp.PICK_HARD, hesp.PICK_SOFT])
@pytest.mark.parametrize("key,n,b,NL,iters", [("cfg0", 3, 1024, 2, 12), ("cfg1a", 4, 2048, 3, 6),
                                              ("cfg1b", 4, 2048, 3, 6), ("cfg2", 3, 1024, 3, 6)])
def test_solver_trajectory_parity(mode, pick, key, n, b, NL, iters):
    spec = W.PLATFORMS[key]
    nb = W.base_count(n)
    rng = np.random.default_rng(mode * 10 + pick + n)
    for start in (np.zeros(nb, np.int8), rng.integers(0, NL, nb).astype(np.int8)):
        seed = 1000 + mode
        sv = S.IterativeSolver(spec, n, b, NL, mode, pick)
        g = sv.solve(start, seed, iters)
        o = V.solve(O.make_platform(spec), n, b, start, NL, mode, pick, seed, iters)
        same_trajectory(g, o)


@pytest.mark.parametrize("mode,pick", [(hesp.SOLVER_ALL, hesp.PICK_HARD), (hesp.SOLVER_CP, hesp.PICK_SOFT)])
def test_solver_trajectory_parity_cfg1_size(mode, pick):
    """8 x 8 tiles (120 base tasks, up to 240 moves per iteration)."""
    spec = W.PLATFORMS["cfg1a"]
    start = W.workload_levels("cfg1", 7, 1)[0]
    sv = S.IterativeSolver(spec, 8, 2048, 3, mode, pick)
    g = sv.solve(start, 9, 3)
    o = V.solve(O.make_platform(spec), 8, 2048, start, 3, mode, pick, 9, 3)
    same_trajectory(g, o)
    assert all(x.chosen is not None for x in g[:-1])


def test_iterative_search_arm_small_budget():
    spec = W.PLATFORMS["cfg1a"]
    log = S.iterative_search(spec, 8, 2048, 3, hesp.SOLVER_ALL, hesp.PICK_HARD, seed=3, budget_s=1.0)
    assert log.best and all(a >= b_ for a, b_ in zip(log.best, log.best[1:]))
    assert all(a <= b_ for a, b_ in zip(log.events, log.events[1:]))
    # the first restart starts from draw 0 of stream 3 and only improves it
    lv0 = W.uniform_levels(3, 0, 1, 120, 3)[0]
    m0 = O.simulate(O.make_platform(spec), 8, 2048, lv0, schedule=False)["makespan"]
    assert log.best[0] <= m0


@pytest.mark.parametrize("mode", [hesp.SOLVER_ALL, hesp.SOLVER_CP, hesp.SOLVER_SHALLOW])
@pytest.mark.parametrize("pick", [hesp.PICK_HARD, hesp.PICK_SOFT])
@pytest.mark.parametrize("key,n", [("cfg1a", 3), ("cfg1b", 3), ("cfg2", 2)])
def test_factor_solver_trajectory_parity(mode, pick, key, n):
    """The solver over partition factors (p = 1/k, k in 1..4, non-dyadic
    moves): GPU trajectories equal the oracle's, from the unsplit partition
    and from a random factor vector."""
    spec = W.PLATFORMS[key]
    nb = W.base_count(n)
    b = 3072
    for start in (np.ones(nb, np.int8), W.uniform_factors(mode * 7 + pick, 0, 1, nb, 4)[0]):
        seed = 2000 + mode
        sv = S.IterativeSolver(spec, n, b, 4, mode, pick, factors=True)
        g = sv.solve(start, seed, 6)
        o = V.solve(O.make_platform(spec), n, b, start, 4, mode, pick, seed, 6, factors=True)
        same_trajectory(g, o)


def test_factor_critical_flags_parity():
    """Critical-path flags of factor candidates (hesp_simulate_factors with
    crit) against the oracle, on 8 x 8 tiles."""
    import torch
    spec = W.PLATFORMS["cfg1a"]
    n, b, C = 8, 3072, 16
    nb = W.base_count(n)
    f = W.uniform_factors(31, 0, C, nb, 4)
    plat = hesp.Platform(spec)
    d_f = torch.from_numpy(f.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * nb)
    crit = torch.zeros(C * nb, dtype=torch.int8, device="cuda")
    ms, st, _ = hesp.simulate_factors(plat, cands, d_f, C, n, 4, b, hesp.alloc_workspace_factors(plat, n, 4, C),
                                      crit=crit)
    torch.cuda.synchronize()
    crit = crit.cpu().numpy().reshape(C, nb)
    pl = O.make_platform(spec)
    for c in range(C):
        flags, m = V.critical_bases(pl, n, b, f[c], factors=True)
        assert int(st[c]) == 0 and int(ms[c]) == m
        assert np.array_equal(crit[c], flags), c
