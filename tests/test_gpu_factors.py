"""GPU parity of the general partition parameter (hesp_simulate_factors
through the C ABI): one-level k-way partitions (Sec. 2.1, p = 1/k) with the
non-dyadic tilings of Fig. 4, against the CPU oracle -- makespans, task
counts and full schedules bit-identical -- on every scheduling policy,
caching policy and link model, plus the equivalences with the dyadic path
and per-candidate error statuses."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1602_05510_b300 import hesp  # noqa: E402
from paper_1602_05510_b300 import workloads as W  # noqa: E402

from test_gpu_sim import links_for  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


def gpu_factors(plat, n, b, factors, max_factor=4, schedule=True, max_tiles=None, task_cap=0, cand_b=None):
    f = np.ascontiguousarray(factors, np.int8)
    C, nb = f.shape
    max_tiles = n if max_tiles is None else max_tiles
    d_f = torch.from_numpy(f.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(n, b if cand_b is None else cand_b, np.arange(C, dtype=np.int64) * nb)
    ws = hesp.alloc_workspace_factors(plat, max_tiles, max_factor, C, task_cap)
    nt = torch.empty(C, dtype=torch.int64, device="cuda")
    ms, st, _ = hesp.simulate_factors(plat, cands, d_f, C, max_tiles, max_factor, b, ws, ntasks=nt, task_cap=task_cap)
    torch.cuda.synchronize()
    out = dict(makespan=ms.cpu().numpy(), status=st.cpu().numpy(), ntasks=nt.cpu().numpy())
    if schedule and (out["status"] == 0).all():
        offs = np.zeros(C + 1, np.int64)
        offs[1:] = np.cumsum(out["ntasks"])
        tot = int(offs[-1])
        sched = (torch.from_numpy(offs[:-1].copy()).cuda(), torch.empty(tot, dtype=torch.int16, device="cuda"),
                 torch.empty(tot, dtype=torch.int64, device="cuda"), torch.empty(tot, dtype=torch.int64, device="cuda"))
        hesp.simulate_factors(plat, cands, d_f, C, max_tiles, max_factor, b, ws, schedule=sched, task_cap=task_cap)
        torch.cuda.synchronize()
        out.update(offs=offs, proc=sched[1].cpu().numpy(), start=sched[2].cpu().numpy(),
                   finish=sched[3].cpu().numpy())
    return out


def check(pl, n, b, factors, g):
    for c in range(factors.shape[0]):
        r = O.simulate_factors(pl, n, b, factors[c])
        assert r["status"] == 0
        assert g["status"][c] == 0, (c, g["status"][c])
        assert g["makespan"][c] == r["makespan"], c
        assert g["ntasks"][c] == r["n_tasks"], c
        if "proc" in g:
            a, e = g["offs"][c], g["offs"][c + 1]
            assert np.array_equal(g["proc"][a:e], r["proc"]), c
            assert np.array_equal(g["start"][a:e], r["start"]), c
            assert np.array_equal(g["finish"][a:e], r["finish"]), c


@pytest.mark.parametrize("key,n", [("cfg0", 3), ("cfg1a", 6), ("cfg1b", 6), ("cfg2", 5), ("cfg4", 4)])
def test_random_factors_parity(key, n):
    b = 3072
    f = W.uniform_factors(11, 0, 40, W.base_count(n), 4)
    spec = W.PLATFORMS[key]
    check(O.make_platform(spec), n, b, f, gpu_factors(hesp.Platform(spec), n, b, f))


def test_full_size_workload_sampled():
    """The benchmark's launch (65,536 candidates of 8 x 8 tiles of 3072,
    factors uniform in 1..4, seed 9) on both platforms; every 1,024th
    against the oracle."""
    n, b, C = W.FACTOR_N, W.FACTOR_B, 65536
    f = W.uniform_factors(9, 0, C, W.base_count(n), W.FACTOR_MAX)
    for key in ("cfg1a", "cfg1b"):
        spec = W.PLATFORMS[key]
        g = gpu_factors(hesp.Platform(spec), n, b, f, schedule=False)
        assert (g["status"] == 0).all()
        pl = O.make_platform(spec)
        for c in range(0, C, 1024):
            r = O.simulate_factors(pl, n, b, f[c], schedule=False)
            assert g["makespan"][c] == r["makespan"] and g["ntasks"][c] == r["n_tasks"], (key, c)


@pytest.mark.parametrize("order,select,cache", [(1, 0, 0), (0, 1, 0), (0, 2, 0), (0, 3, 0), (1, 3, 0),
                                                (0, 0, 1), (0, 0, 2), (1, 2, 1)])
def test_policies_parity(order, select, cache):
    n, b = 5, 3072
    f = W.uniform_factors(21 + order * 4 + select, 0, 24, W.base_count(n), 4)
    seed = 0x5555 + 17 * select
    for key in ("cfg1a", "cfg2"):
        spec = W.PLATFORMS[key]
        links = links_for(spec) if cache == 1 else None
        plat = hesp.Platform(spec, order=order, select=select, rp_seed=seed, cache=cache, links=links)
        pl = O.make_platform(spec, order=order, select=select, rp_seed=seed, cache=cache, links=links)
        check(pl, n, b, f, gpu_factors(plat, n, b, f))


def test_factors_one_two_equal_levels_zero_one():
    """Factor 2 is the dyadic level-1 partition and factor 1 keeps the base
    task: hesp_simulate_factors and hesp_simulate_batch agree exactly."""
    n, b, C = 8, 2048, 256
    lv = W.uniform_levels(3, 0, C, W.base_count(n), 2)
    for key in ("cfg1a", "cfg1b"):
        plat = hesp.Platform(W.PLATFORMS[key])
        g = gpu_factors(plat, n, b, lv + 1, max_factor=2)
        d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
        cands = hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * W.base_count(n))
        ms, st, _ = hesp.simulate_batch(plat, cands, d_lv, C, n, 1, hesp.alloc_workspace(plat, n, 1, C))
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all() and (g["status"] == 0).all()
        assert np.array_equal(ms.cpu().numpy(), g["makespan"])


def _closed_tasks(n, f):
    cnt = {0: lambda k: k * (k + 1) * (k + 2) // 6, 1: lambda k: k * k * (k + 1) // 2,
           2: lambda k: k * k * (k + 1) // 2, 3: lambda k: k ** 3}
    return sum(cnt[int(op)](int(k)) for op, k in zip(O.base_ops(n), f))


def test_single_tile_every_factor_and_max_tiles():
    plat = hesp.Platform(W.PLATFORMS["cfg1a"])
    pl = O.make_platform(W.PLATFORMS["cfg1a"])
    f = np.array([[1], [2], [3], [4]], np.int8)
    check(pl, 1, 3072, f, gpu_factors(plat, 1, 3072, f))
    # 24 x 24 tiles against the oracle; the largest matrix (64 x 64 tiles,
    # 299,520 atoms) against the closed-form task count
    fz = W.uniform_factors(5, 0, 1, W.base_count(24), 4)
    g = gpu_factors(plat, 24, 3072, fz, schedule=False)
    r = O.simulate_factors(pl, 24, 3072, fz[0], schedule=False)
    assert g["status"][0] == 0 and g["makespan"][0] == r["makespan"]
    fz = W.uniform_factors(6, 0, 1, W.base_count(64), 4)
    g = gpu_factors(plat, 64, 3072, fz, schedule=False)
    assert g["status"][0] == 0 and g["makespan"][0] > 0
    assert g["ntasks"][0] == _closed_tasks(64, fz[0])


def test_bad_candidates_get_status():
    plat = hesp.Platform(W.PLATFORMS["cfg1a"])
    n, nb = 3, W.base_count(3)
    good = np.full((1, nb), 3, np.int8)
    # 3 does not divide 2048: every candidate of b = 2048 with a factor 3 is refused
    g = gpu_factors(plat, n, 2048, good, schedule=False)
    assert g["status"][0] == hesp.HESP_ERR_ARG and g["makespan"][0] == -1
    # a factor out of range, and a candidate whose b is not the launch's
    bad = np.ones((3, nb), np.int8)
    bad[0, 2] = 0
    bad[1, 4] = 5
    g = gpu_factors(plat, n, 3072, bad, schedule=False)
    assert g["status"][0] == hesp.HESP_ERR_ARG and g["status"][1] == hesp.HESP_ERR_ARG and g["status"][2] == 0
    g = gpu_factors(plat, n, 3072, np.ones((1, nb), np.int8), schedule=False, cand_b=1536)
    assert g["status"][0] == hesp.HESP_ERR_ARG
    # a task cap below the DAG size: HESP_ERR_CAPACITY for that candidate only
    f = np.ones((2, nb), np.int8)
    f[0, :] = 4
    g = gpu_factors(plat, n, 3072, f, schedule=False, task_cap=20)
    assert g["status"][0] == hesp.HESP_ERR_CAPACITY and g["status"][1] == 0
    # an empty batch and an unsupported factor bound
    ws = hesp.alloc_workspace_factors(plat, n, 4, 1)
    cands = hesp.cands_tensor(n, 3072, np.zeros(1, np.int64))
    d_f = torch.ones(nb, dtype=torch.int8, device="cuda")
    hesp.simulate_factors(plat, cands, d_f, 0, n, 4, 3072, ws)
    with pytest.raises(hesp.HespError):
        hesp.simulate_factors(plat, cands, d_f, 1, n, 5, 3072, ws)


@pytest.mark.parametrize("order,select,cache", [(0, 0, 0), (1, 0, 1)])
def test_32x32_tiles_with_schedules(order, select, cache):
    """The search workload's size: 32 x 32 tiles (5,984 base tasks, ~140,000
    tasks per candidate) with factors 1..4 on 32 CPU + 2 GPU-type
    processors (two accelerator memories, more than 32 processors), full
    schedules against the oracle."""
    spec = W.PLATFORMS["cfg4"]
    n, b = 32, 3072
    f = W.uniform_factors(13 + order, 0, 2, W.base_count(n), 4)
    plat = hesp.Platform(spec, order=order, select=select, cache=cache)
    pl = O.make_platform(spec, order, select, cache=cache)
    check(pl, n, b, f, gpu_factors(plat, n, b, f))
