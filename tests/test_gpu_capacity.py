"""GPU parity of finite accelerator memories (hesp_platform_set_capacity)
against the CPU oracle: makespans and full schedules bit-identical under
every task order, EFT-P / EIT-P, every caching policy, one and two
accelerator memories, with the hand-derived examples of the oracle's pins,
keep / reuse launches, and the refused combinations."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1602_05510_b300 import hesp  # noqa: E402
from paper_1602_05510_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

MB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


def run(plat, n, b, lv, max_level=None):
    lv = np.ascontiguousarray(lv, np.int8)
    C, nb = lv.shape
    L = int(lv.max()) if max_level is None else max_level
    d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * nb)
    ws = hesp.alloc_workspace(plat, n, L, C)
    dag = hesp.Dag(n, b, L)
    cnt = np.array([dag.count_tasks(lv[c])[0] for c in range(C)], np.int64)
    offs = np.zeros(C + 1, np.int64)
    offs[1:] = np.cumsum(cnt)
    tot = int(offs[-1])
    sched = (torch.from_numpy(offs[:-1].copy()).cuda(), torch.empty(tot, dtype=torch.int16, device="cuda"),
             torch.empty(tot, dtype=torch.int64, device="cuda"), torch.empty(tot, dtype=torch.int64, device="cuda"))
    ms, st, _ = hesp.simulate_batch(plat, cands, d_lv, C, n, L, ws, schedule=sched)
    torch.cuda.synchronize()
    return dict(makespan=ms.cpu().numpy(), status=st.cpu().numpy(), offs=offs, proc=sched[1].cpu().numpy(),
                start=sched[2].cpu().numpy(), finish=sched[3].cpu().numpy())


def check(pl, n, b, lv, g):
    """Parity of every candidate; returns the atoms the oracle evicted."""
    evicted = 0
    for c in range(lv.shape[0]):
        r = O.simulate(pl, n, b, lv[c])
        evicted += r["evicted"]
        assert g["status"][c] == r["status"], (c, g["status"][c], r["status"])
        if r["status"] != 0:
            continue
        assert g["makespan"][c] == r["makespan"], c
        a, e = g["offs"][c], g["offs"][c + 1]
        assert np.array_equal(g["proc"][a:e], r["proc"]), c
        assert np.array_equal(g["start"][a:e], r["start"]), c
        assert np.array_equal(g["finish"][a:e], r["finish"]), c
    return evicted


B = 256
ATOM = B * B * 8


def two_mem_spec(procs):
    """The oracle pins' platform: GPU chol / trsm / syrk 10 / 20 / 30 us, CPU ten
    times slower, messages of k atoms 1000 + k ns."""
    ty = W.CPU_TYPE
    ovr = ((0, 1, B, 10_000), (1, 1, B, 20_000), (2, 1, B, 30_000),
           (0, 0, B, 100_000), (1, 0, B, 200_000), (2, 0, B, 300_000))
    return types.SimpleNamespace(name="pin", n_mem=2, types=(ty, ty), procs=tuple(procs), xfer_latency_ns=1000,
                                 bytes_per_elem=8, bw_bytes_per_ns=ATOM, exec_overrides=ovr)


def test_hand_derived_examples():
    lv = np.zeros((1, 4), np.int8)
    g = run(hesp.Platform(two_mem_spec([(1, 1)]), capacity={1: 2 * ATOM}), 2, B, lv, 0)
    assert g["status"][0] == 0 and g["makespan"][0] == 73_003
    assert list(g["finish"]) == [11_001, 32_002, 63_003, 73_003]
    g = run(hesp.Platform(two_mem_spec([(1, 1)]), capacity={1: ATOM}), 2, B, lv, 0)
    assert g["status"][0] == hesp.HESP_ERR_CAPACITY and g["makespan"][0] == -1
    g = run(hesp.Platform(two_mem_spec([(0, 0), (1, 1)]), capacity={1: ATOM}), 2, B, lv, 0)
    assert g["status"][0] == 0 and g["makespan"][0] == 523_003
    assert list(g["proc"]) == [1, 0, 0, 1] and list(g["finish"]) == [11_001, 212_002, 512_002, 523_003]


@pytest.mark.parametrize("cap_mb", [40, 100, 300, 700])
@pytest.mark.parametrize("order,select,cache", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 0, 2)])
def test_random_candidates_parity(cap_mb, order, select, cache):
    spec = W.PLATFORMS["cfg1a"]
    n, b = 8, 2048
    lv = W.workload_levels("cfg1", 700 + cap_mb, 10)
    plat = hesp.Platform(spec, order=order, select=select, cache=cache, capacity={1: cap_mb * MB})
    pl = O.make_platform(spec, order, select, cache=cache, capacity={1: cap_mb * MB})
    evicted = check(pl, n, b, lv, run(plat, n, b, lv))
    if cap_mb <= 300:
        assert evicted > 0  # the memory is really full


@pytest.mark.parametrize("key,n,b", [("cfg2", 6, 1024), ("cfg4", 5, 2048)])
def test_two_accelerator_memories(key, n, b):
    spec = W.PLATFORMS[key]
    lv = np.random.default_rng(8).integers(0, 3, (12, W.base_count(n))).astype(np.int8)
    for caps in ({1: 20 * MB}, {1: 20 * MB, 2: 60 * MB}, {2: 8 * MB}):
        plat = hesp.Platform(spec, capacity=caps)
        check(O.make_platform(spec, capacity=caps), n, b, lv, run(plat, n, b, lv))


def test_keep_and_reuse_with_capacity():
    n, b, C = 8, 2048, 512
    lv = W.workload_levels("cfg1", 5000, C)
    d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * W.base_count(n))
    ws = hesp.alloc_workspace_kept(n, 2, C)
    hesp.dag_build_kept(cands, d_lv, C, n, 2, ws)
    for caps in ({1: 64 * MB}, {1: 256 * MB}):
        plat = hesp.Platform(W.PLATFORMS["cfg1a"], capacity=caps)
        ms, st, _ = hesp.simulate_batch_reuse(plat, cands, d_lv, C, n, 2, ws)
        ms2, st2, _ = hesp.simulate_batch(plat, cands, d_lv, C, n, 2, hesp.alloc_workspace(plat, n, 2, C))
        torch.cuda.synchronize()
        assert torch.equal(st, st2) and torch.equal(ms, ms2)
        assert int((st == 0).sum()) == C


def test_refused_combinations():
    spec = W.PLATFORMS["cfg1a"]
    n = 3
    lv = torch.zeros(W.base_count(n), dtype=torch.int8, device="cuda")
    cands = hesp.cands_tensor(n, 3072, np.zeros(1, np.int64))
    for sel in (2, 3):
        plat = hesp.Platform(spec, select=sel, capacity={1: 64 * MB})
        with pytest.raises(hesp.HespError):
            hesp.simulate_batch(plat, cands, lv, 1, n, 0, hesp.alloc_workspace(plat, n, 0, 1))
    plat = hesp.Platform(spec, capacity={1: 64 * MB})
    with pytest.raises(hesp.HespError):
        hesp.simulate_factors(plat, cands, torch.ones_like(lv), 1, n, 4, 3072, hesp.alloc_workspace_factors(plat, n, 4, 1))
    with pytest.raises(hesp.HespError):
        hesp.Platform(spec, capacity={0: 64 * MB})  # host memory is unbounded


def test_capacity_workload_full_launch_sampled():
    """The benchmark's finite-memory launch: 65,536 candidates of 8 x 8 tiles
    on 12 CPU + 1 GPU-type with 256 MB of GPU memory; every 512th candidate
    against the oracle."""
    n, b, C = 8, 2048, 65536
    nb = W.base_count(n)
    plat = hesp.Platform(W.PLATFORMS["cfg1a"], capacity={1: 256 * MB})
    cands = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    levels = torch.empty(C * nb, dtype=torch.int8, device="cuda")
    hesp.generate_candidates(hesp.GEN_UNIFORM, 1, 0, C, n, b, 3, levels, cands)
    ms, st, nt = hesp.simulate_batch(plat, cands, levels, C, n, 2, hesp.alloc_workspace(plat, n, 2, C),
                                     ntasks=torch.empty(C, dtype=torch.int64, device="cuda"))
    torch.cuda.synchronize()
    ms, st, nt = ms.cpu().numpy(), st.cpu().numpy(), nt.cpu().numpy()
    assert (st == 0).all()
    lv = W.uniform_levels(1, 0, C, nb, 3)
    pl = O.make_platform(W.PLATFORMS["cfg1a"], capacity={1: 256 * MB})
    for c in range(0, C, 512):
        r = O.simulate(pl, n, b, lv[c], schedule=False)
        assert ms[c] == r["makespan"] and nt[c] == r["n_tasks"], c
