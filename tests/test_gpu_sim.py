"""GPU parity of the batched simulator (hesp_simulate_batch through the C ABI)
against the CPU oracle: makespans, per-task processors, start and finish times
must be bit-identical (int64 ns, fixed tie-breaking), on every workload shape,
at oracle-sized samples and at the full 65,536-candidate launch the benchmark
times, plus edge cases and per-candidate error statuses."""
import dataclasses
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1602_05510_b300 import hesp  # noqa: E402
from paper_1602_05510_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


def gpu_sim(spec, n, b, levels, max_level=None, schedule=False, max_tiles=None, ws_cands=None, task_cap=0):
    """Run one batch of candidates of the same (n, b) on the GPU."""
    levels = np.ascontiguousarray(levels, np.int8)
    C, nb = levels.shape
    max_level = int(levels.max()) if max_level is None else max_level
    max_tiles = n if max_tiles is None else max_tiles
    plat = hesp.Platform(spec)
    lv = torch.from_numpy(levels.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * nb)
    ws = hesp.alloc_workspace(plat, max_tiles, max_level, C if ws_cands is None else ws_cands, task_cap,
                              max_bytes=8 << 30)
    ntasks = torch.empty(C, dtype=torch.int64, device="cuda")
    sched = None
    offs = None
    if schedule:
        dag = hesp.Dag(n, b, max(max_level, 0))
        cnt = np.array([dag.count_tasks(levels[c])[0] for c in range(C)], np.int64)
        offs = np.zeros(C + 1, np.int64)
        offs[1:] = np.cumsum(cnt)
        tot = int(offs[-1])
        sched = (torch.from_numpy(offs[:-1].copy()).cuda(), torch.empty(tot, dtype=torch.int16, device="cuda"),
                 torch.empty(tot, dtype=torch.int64, device="cuda"), torch.empty(tot, dtype=torch.int64, device="cuda"))
    ms, st, nt = hesp.simulate_batch(plat, cands, lv, C, max_tiles, max_level, ws, ntasks=ntasks, schedule=sched,
                                     task_cap=task_cap)
    torch.cuda.synchronize()
    out = dict(makespan=ms.cpu().numpy(), status=st.cpu().numpy(), ntasks=nt.cpu().numpy())
    if schedule:
        out.update(offs=offs, proc=sched[1].cpu().numpy(), start=sched[2].cpu().numpy(),
                   finish=sched[3].cpu().numpy())
    return out


def check_parity(spec, n, b, levels, g, idx=None, schedule=True):
    pl = O.make_platform(spec)
    idx = range(levels.shape[0]) if idx is None else idx
    for c in idx:
        r = O.simulate(pl, n, b, levels[c], schedule=schedule)
        assert r["status"] == 0
        assert g["status"][c] == 0, (c, g["status"][c])
        assert g["makespan"][c] == r["makespan"], c
        assert g["ntasks"][c] == r["n_tasks"], c
        if schedule and "proc" in g:
            a, e = g["offs"][c], g["offs"][c + 1]
            assert np.array_equal(g["proc"][a:e], r["proc"]), c
            assert np.array_equal(g["start"][a:e], r["start"]), c
            assert np.array_equal(g["finish"][a:e], r["finish"]), c


def test_worked_examples_on_gpu():
    for key in ("n2_b1024_all_level0_cpu4_gpu1", "n1_b1024_chol_level1_cpu4_gpu1"):
        e = GOLD[key]
        g = gpu_sim(W.PLATFORMS[e["platform"]], e["n"], e["b"], np.array([e["levels"]]), schedule=True)
        assert g["makespan"][0] == e["makespan"]
        assert g["proc"].tolist() == e["proc"] and g["finish"].tolist() == e["finish"]
    for key, ncpu in (("n2_b1024_cpu1_gpu1_overrides", 1), ("n3_b1024_cpu2_gpu1_overrides", 2)):
        e = GOLD[key]
        spec = dataclasses.replace(W.cpu_gpu_platform(ncpu, 1), exec_overrides=tuple(tuple(x) for x in e["overrides"]))
        g = gpu_sim(spec, e["n"], e["b"], np.array([e["levels"]]), schedule=True)
        assert g["makespan"][0] == e["makespan"]
        assert g["proc"].tolist() == e["proc"]
        assert g["start"].tolist() == e["start"] and g["finish"].tolist() == e["finish"]


def test_cfg0_exhaustive_all_1024():
    lv = W.workload_levels("cfg0")
    g = gpu_sim(W.PLATFORMS["cfg0"], 3, 1024, lv, max_level=1, schedule=True)
    check_parity(W.PLATFORMS["cfg0"], 3, 1024, lv, g)


@pytest.mark.parametrize("key", ["cfg1a", "cfg1b"])
def test_cfg1_sample_with_schedules(key):
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(65536, 192, replace=False))
    lv = np.concatenate([W.workload_levels("cfg1", int(i), 1) for i in idx])
    g = gpu_sim(W.PLATFORMS[key], 8, 2048, lv, max_level=2, schedule=True)
    check_parity(W.PLATFORMS[key], 8, 2048, lv, g)


@pytest.mark.parametrize("key", ["cfg1a", "cfg1b"])
def test_cfg1_full_launch_sampled(key):
    """The whole 65,536-candidate batch in one launch (the benchmark's launch
    configuration); sampled candidates checked against the oracle, the rest
    by properties that hold at any size."""
    lv = W.workload_levels("cfg1")
    g = gpu_sim(W.PLATFORMS[key], 8, 2048, lv, max_level=2)
    assert (g["status"] == 0).all()
    dag = hesp.Dag(8, 2048, 2)
    rng = np.random.default_rng(5)
    for c in rng.choice(65536, 200, replace=False):
        assert g["ntasks"][c] == dag.count_tasks(lv[c])[0]
    assert (g["makespan"] > 0).all()
    idx = np.sort(rng.choice(65536, 48, replace=False))
    check_parity(W.PLATFORMS[key], 8, 2048, lv, g, idx=idx, schedule=False)


def test_device_generation_matches_host():
    n = 8
    nb = W.base_count(n)
    lv = torch.empty(4096 * nb, dtype=torch.int8, device="cuda")
    cands = torch.empty(4096 * 16, dtype=torch.uint8, device="cuda")
    hesp.generate_candidates(hesp.GEN_UNIFORM, 1, 1000, 4096, n, 2048, 3, lv, cands)
    torch.cuda.synchronize()
    assert np.array_equal(lv.cpu().numpy().reshape(4096, nb), W.uniform_levels(1, 1000, 4096, nb, 3))
    c = cands.cpu().numpy().view(hesp.CAND_DTYPE)
    assert (c["n_tiles"] == n).all() and (c["b"] == 2048).all()
    assert np.array_equal(c["level_offset"], np.arange(4096) * nb)
    lv0 = torch.empty(1024 * 10, dtype=torch.int8, device="cuda")
    hesp.generate_candidates(hesp.GEN_EXHAUSTIVE, 0, 0, 1024, 3, 1024, 2, lv0)
    torch.cuda.synchronize()
    assert np.array_equal(lv0.cpu().numpy().reshape(1024, 10), W.exhaustive_levels(10))
    lv4 = torch.empty(64 * 5984, dtype=torch.int8, device="cuda")
    hesp.generate_candidates(hesp.GEN_UNIFORM, 4, 0, 64, 32, 2048, 4, lv4)
    torch.cuda.synchronize()
    assert np.array_equal(lv4.cpu().numpy().reshape(64, 5984), W.uniform_levels(4, 0, 64, 5984, 4))


def test_uneven_generation_and_parity():
    C = 256
    n, b, off, lvh = W.uneven_candidates(2, 0, C)
    cands = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    lv = torch.empty(int(off[-1]) + 100, dtype=torch.int8, device="cuda")
    used = torch.zeros(1, dtype=torch.int64, device="cuda")
    hesp.generate_uneven(2, 0, C, cands, lv, used)
    torch.cuda.synchronize()
    assert int(used.item()) == int(off[-1])
    cd = cands.cpu().numpy().view(hesp.CAND_DTYPE)
    assert np.array_equal(cd["n_tiles"], n) and np.array_equal(cd["b"], b)
    assert np.array_equal(cd["level_offset"], off[:-1])
    assert np.array_equal(lv.cpu().numpy()[:off[-1]], lvh)
    # simulate the ragged batch and check a budget of small and large ones
    spec = W.PLATFORMS["cfg2"]
    plat = hesp.Platform(spec)
    ws = hesp.alloc_workspace(plat, 32, 2, C)
    ntasks = torch.empty(C, dtype=torch.int64, device="cuda")
    ms, st, nt = hesp.simulate_batch(plat, cands, lv, C, 32, 2, ws, ntasks=ntasks)
    torch.cuda.synchronize()
    ms, st, nt = ms.cpu().numpy(), st.cpu().numpy(), nt.cpu().numpy()
    assert (st == 0).all()
    pl = O.make_platform(spec)
    order = np.argsort(nt)
    pick = list(order[:24]) + list(order[-3:]) + list(order[C // 2:C // 2 + 6])
    for c in pick:
        r = O.simulate(pl, int(n[c]), int(b[c]), lvh[off[c]:off[c + 1]], schedule=False)
        assert r["makespan"] == ms[c] and r["n_tasks"] == nt[c], c


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_single_tile_every_level(level):
    lv = np.array([[level]], np.int8)
    for key in ("cfg0", "cfg2", "cfg1b"):
        g = gpu_sim(W.PLATFORMS[key], 1, 2048, lv, schedule=True)
        check_parity(W.PLATFORMS[key], 1, 2048, lv, g)


def test_more_than_32_processors_and_four_levels():
    rng = np.random.default_rng(3)
    lv = rng.integers(0, 4, (24, W.base_count(5))).astype(np.int8)
    g = gpu_sim(W.PLATFORMS["cfg4"], 5, 2048, lv, max_level=3, schedule=True)
    check_parity(W.PLATFORMS["cfg4"], 5, 2048, lv, g)
    spec = W.cpu_gpu_platform(60, 3)   # 63 processors, 4 memories
    g = gpu_sim(spec, 4, 1024, lv[:, :W.base_count(4)], max_level=3, schedule=True)
    check_parity(spec, 4, 1024, lv[:, :W.base_count(4)], g)


def test_single_processor_and_identical_processors():
    rng = np.random.default_rng(8)
    lv = rng.integers(0, 3, (16, W.base_count(4))).astype(np.int8)
    for spec in (W.single_cpu_platform(), W.PlatformSpec("id3", 1, (W.CPU_TYPE,), ((0, 0),) * 3)):
        g = gpu_sim(spec, 4, 512, lv, max_level=2, schedule=True)
        check_parity(spec, 4, 512, lv, g)


def test_workspace_smaller_than_batch():
    """Fewer arenas than candidates: warps pull candidates until done."""
    lv = W.workload_levels("cfg1", 0, 300)
    g = gpu_sim(W.PLATFORMS["cfg1a"], 8, 2048, lv, max_level=2, ws_cands=7)
    check_parity(W.PLATFORMS["cfg1a"], 8, 2048, lv, g, idx=range(0, 300, 37), schedule=False)


def test_bad_candidates_get_status_not_fault():
    spec = W.PLATFORMS["cfg0"]
    plat = hesp.Platform(spec)
    nb = 10
    lvh = np.zeros((4, nb), np.int8)
    lvh[1, 3] = 3      # above max_level = 2
    lvh[2, 0] = -1     # negative
    lv = torch.from_numpy(lvh.reshape(-1).copy()).cuda()
    a = np.zeros(6, hesp.CAND_DTYPE)
    a["n_tiles"] = [3, 3, 3, 3, 4, 3]
    a["b"] = [1024, 1024, 1024, 1000, 1024, 1]
    a["level_offset"] = [0, nb, 2 * nb, 3 * nb, 0, 0]
    lvh[0, 0] = 0
    cands = torch.from_numpy(a.view(np.uint8).copy()).cuda()
    ws = hesp.alloc_workspace(plat, 3, 2, 6)
    ms, st, _ = hesp.simulate_batch(plat, cands, lv, 6, 3, 2, ws)
    torch.cuda.synchronize()
    st = st.cpu().numpy().tolist()
    # b = 1 with every level 0 is a valid (tiny) problem
    assert st == [0, -1, -1, -1, -1, 0]
    with pytest.raises(hesp.HespError):
        hesp.simulate_batch(plat, cands, lv, 6, 3, 2, ws[:100])


def test_task_cap_reports_capacity_and_keeps_others_exact():
    lv = W.workload_levels("cfg1", 0, 96)
    spec = W.PLATFORMS["cfg1a"]
    plat = hesp.Platform(spec)
    C = lv.shape[0]
    ws = hesp.alloc_workspace(plat, 8, 2, C, task_cap=2300)
    nt = torch.empty(C, dtype=torch.int64, device="cuda")
    ms, st, _ = hesp.simulate_batch(plat, hesp.cands_tensor(8, 2048, np.arange(C) * 120),
                                    torch.from_numpy(lv.reshape(-1).copy()).cuda(), C, 8, 2, ws, ntasks=nt,
                                    task_cap=2300)
    torch.cuda.synchronize()
    st, ms = st.cpu().numpy(), ms.cpu().numpy()
    dag = hesp.Dag(8, 2048, 2)
    T = np.array([dag.count_tasks(r)[0] for r in lv])
    assert ((T > 2300) == (st == -2)).all() and (st[T <= 2300] == 0).all()
    assert (T > 2300).any() and (T <= 2300).any()
    pl = O.make_platform(spec)
    for c in np.nonzero(T <= 2300)[0][:12]:
        assert O.simulate(pl, 8, 2048, lv[c], schedule=False)["makespan"] == ms[c]


def test_cfg4_full_size_candidates():
    """n = 32 tiles, levels 0..3 (about 8e5 tasks per candidate) on the
    32 CPU + 2 GPU platform, checked against the oracle."""
    lv = W.workload_levels("cfg4", 0, 2)
    g = gpu_sim(W.PLATFORMS["cfg4"], 32, 2048, lv, max_level=3, task_cap=1 << 20)
    check_parity(W.PLATFORMS["cfg4"], 32, 2048, lv, g, schedule=False)


def links_for(spec):
    links = {(0, 1): (20000, 6), (1, 0): (15000, 9)}
    if spec.n_mem > 2:
        links.update({(1, 2): (1000, 50), (2, 1): (1500, 40), (0, 2): (9000, 12), (2, 0): (4000, 30)})
    return links


def policy_parity(order, select, cache=0, with_links=False):
    seed = 0x8000000000000000 + 12345 * (order + 1)
    cases = [("cfg0", 3, 1024, W.workload_levels("cfg0")[::8], 1),
             ("cfg1a", 8, 2048, W.workload_levels("cfg1", 300, 48), 2),
             ("cfg1b", 8, 2048, W.workload_levels("cfg1", 900, 48), 2),
             ("cfg2", 6, 512, np.random.default_rng(1).integers(0, 3, (24, W.base_count(6))).astype(np.int8), 2),
             ("cfg4", 5, 2048, np.random.default_rng(2).integers(0, 4, (16, W.base_count(5))).astype(np.int8), 3)]
    for key, n, b, lv, L in cases:
        spec = W.PLATFORMS[key]
        links = links_for(spec) if with_links and spec.n_mem > 1 else None
        plat = hesp.Platform(spec, order=order, select=select, rp_seed=seed, cache=cache, links=links)
        C, nb = lv.shape
        d_lv = torch.from_numpy(np.ascontiguousarray(lv).reshape(-1).copy()).cuda()
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
        ms, st = ms.cpu().numpy(), st.cpu().numpy()
        proc, start, fin = (x.cpu().numpy() for x in sched[1:])
        pl = O.make_platform(spec, order=order, select=select, rp_seed=seed, cache=cache, links=links)
        for c in range(C):
            r = O.simulate(pl, n, b, lv[c])
            assert st[c] == 0 and ms[c] == r["makespan"], (key, c)
            a, e = offs[c], offs[c + 1]
            assert np.array_equal(proc[a:e], r["proc"]) and np.array_equal(start[a:e], r["start"]), (key, c)
            assert np.array_equal(fin[a:e], r["finish"]), (key, c)


@pytest.mark.parametrize("order,select", [(0, 1), (1, 0), (1, 1), (0, 2), (0, 3), (1, 2), (1, 3)])
def test_policies_parity(order, select):
    """PL task order and the EIT-P, F-P and R-P processor choices (Sec. 2.1)
    against the oracle: schedules bit-exact on every workload shape."""
    policy_parity(order, select)


@pytest.mark.parametrize("cache", [1, 2])
@pytest.mark.parametrize("order,select", [(0, 0), (1, 0), (0, 2), (1, 3)])
def test_cache_policies_parity(cache, order, select):
    """Write-through and write-around caching (Sec. 2.1) against the oracle,
    with several task orders and processor choices: schedules bit-exact."""
    policy_parity(order, select, cache)


@pytest.mark.parametrize("cache", [0, 1, 2])
@pytest.mark.parametrize("order,select", [(0, 0), (1, 2)])
def test_link_costs_parity(cache, order, select):
    """Per-link transfer costs (asymmetric, a fast GPU-GPU link) against the
    oracle: schedules bit-exact."""
    policy_parity(order, select, cache, with_links=True)


def test_maximum_tiles_and_empty_batch():
    """The largest matrix the ABI allows (64 x 64 tiles, 45,760 base tasks),
    unsplit and with some splits, against the oracle; and an empty batch,
    which launches nothing and succeeds."""
    nb = W.base_count(hesp.MAX_TILES)
    lv = np.zeros((2, nb), np.int8)
    lv[1, ::97] = 1
    for key in ("cfg1a", "cfg1b"):
        g = gpu_sim(W.PLATFORMS[key], hesp.MAX_TILES, 512, lv, max_level=1)
        check_parity(W.PLATFORMS[key], hesp.MAX_TILES, 512, lv, g, schedule=False)
    plat = hesp.Platform(W.PLATFORMS["cfg0"])
    ws = hesp.alloc_workspace(plat, 3, 1, 1)
    empty = torch.empty(0, dtype=torch.int8, device="cuda")
    ms, st, _ = hesp.simulate_batch(plat, hesp.cands_tensor(3, 1024, np.zeros(0, np.int64)), empty, 0, 3, 1, ws)
    assert ms.numel() == 0 and st.numel() == 0


def test_keep_and_reuse_equal_separate_simulations():
    """One DAG build, several platforms: hesp_simulate_batch_keep on the CPU+GPU
    platform, then hesp_simulate_batch_reuse on big.LITTLE, on the first
    platform again and on a PL / EIT-P platform, each equal to a separate
    hesp_simulate_batch; a candidate whose levels changed after the keep call
    gets HESP_ERR_STATE, one whose build failed keeps the build's status."""
    C, nb = 300, 120
    lvh = W.workload_levels("cfg1", 4000, C)
    lvh[7, 5] = 3  # above max_level: the build fails (HESP_ERR_ARG)
    lv = torch.from_numpy(lvh.reshape(-1).copy()).cuda()
    order = np.random.default_rng(0).permutation(C).astype(np.int64)  # any candidate order works
    cands = hesp.cands_tensor(8, 2048, order * nb)
    ws = hesp.alloc_workspace_kept(8, 2, C)
    specs = [hesp.Platform(W.PLATFORMS["cfg1a"]), hesp.Platform(W.PLATFORMS["cfg1b"]),
             hesp.Platform(W.PLATFORMS["cfg1a"]), hesp.Platform(W.PLATFORMS["cfg2"], order=1, select=1)]
    for i, plat in enumerate(specs):
        f = hesp.simulate_batch_keep if i == 0 else hesp.simulate_batch_reuse
        nt = torch.empty(C, dtype=torch.int64, device="cuda")
        ms, st, _ = f(plat, cands, lv, C, 8, 2, ws, ntasks=nt)
        ref_ws = hesp.alloc_workspace(plat, 8, 2, C)
        nt2 = torch.empty(C, dtype=torch.int64, device="cuda")
        ms2, st2, _ = hesp.simulate_batch(plat, cands, lv, C, 8, 2, ref_ws, ntasks=nt2)
        torch.cuda.synchronize()
        assert torch.equal(st, st2) and torch.equal(ms, ms2) and torch.equal(nt[st == 0], nt2[st2 == 0]), i
        bad = int(np.nonzero(order == 7)[0][0])
        assert int(st[bad].item()) == -1 and int((st == 0).sum().item()) == C - 1
    # change two candidates' levels after the keep call
    lv2 = lv.clone()
    lv2[3 * nb + 10] = (lv2[3 * nb + 10] + 1) % 3
    lv2[11 * nb + 0] = (lv2[11 * nb + 0] + 1) % 3
    ms, st, _ = hesp.simulate_batch_reuse(specs[1], cands, lv2, C, 8, 2, ws)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    changed = {int(np.nonzero(order == 3)[0][0]), int(np.nonzero(order == 11)[0][0])}
    for c in range(C):
        if c in changed:
            assert st[c] == -5
        elif order[c] == 7:
            assert st[c] == -1
        else:
            assert st[c] == 0
    with pytest.raises(hesp.HespError):
        hesp.simulate_batch_keep(specs[0], cands, lv, C, 8, 2, ws[:ws.numel() // 2])


def test_cfg2_full_ragged_launch_sampled():
    """The full 16,384-candidate ragged batch (n 4..32, b 512..2048), ordered
    largest DAG first as the benchmark runs it: every candidate succeeds, task
    counts match the closed forms, and a sample across sizes matches the
    oracle."""
    C = 16384
    cands = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    lv = torch.empty(C * W.base_count(32), dtype=torch.int8, device="cuda")
    used = torch.zeros(1, dtype=torch.int64, device="cuda")
    hesp.generate_uneven(2, 0, C, cands, lv, used)
    scands, perm = hesp.sort_cands_by_size(cands, lv, C)
    spec = W.PLATFORMS["cfg2"]
    plat = hesp.Platform(spec)
    ws = hesp.alloc_workspace(plat, 32, 2, C, max_bytes=16 << 30)
    nt = torch.empty(C, dtype=torch.int64, device="cuda")
    ms, st, _ = hesp.simulate_batch(plat, scands, lv, C, 32, 2, ws, ntasks=nt)
    torch.cuda.synchronize()
    ms, st, nt, perm = ms.cpu().numpy(), st.cpu().numpy(), nt.cpu().numpy(), perm.cpu().numpy()
    assert (st == 0).all()
    assert (np.diff(np.minimum(nt >> 4, 65535)) <= 0).all()  # largest first, in buckets of 16 tasks
    assert np.array_equal(np.sort(perm), np.arange(C))
    n, b, off, lvh = W.uneven_candidates(2, 0, C)
    pl = O.make_platform(spec)
    order = np.argsort(nt)
    pick = list(order[:8]) + list(order[C // 2:C // 2 + 6]) + list(order[-3:])
    for i in pick:
        c = int(perm[i])  # original candidate index
        r = O.simulate(pl, int(n[c]), int(b[c]), lvh[off[c]:off[c + 1]], schedule=False)
        assert r["makespan"] == ms[i] and r["n_tasks"] == nt[i], (i, c)


def test_cfg3_full_label_launch_sampled():
    """A full 65,536-candidate labelling launch of the surrogate workload
    (16 x 16 tiles, levels {0,1,2}, 16 CPU + 2 GPU): all succeed, sampled
    candidates match the oracle."""
    C, n, b = 65536, 16, 2048
    nb = W.base_count(n)
    lv = torch.empty(C * nb, dtype=torch.int8, device="cuda")
    hesp.generate_candidates(hesp.GEN_UNIFORM, 3, 0, C, n, b, 3, lv)
    spec = W.PLATFORMS["cfg3"]
    plat = hesp.Platform(spec)
    ws = hesp.alloc_workspace(plat, n, 2, C, max_bytes=16 << 30)
    ms, st, _ = hesp.simulate_batch(plat, hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * nb), lv, C, n, 2, ws)
    torch.cuda.synchronize()
    ms, st = ms.cpu().numpy(), st.cpu().numpy()
    assert (st == 0).all()
    pl = O.make_platform(spec)
    idx = np.sort(np.random.default_rng(3).choice(C, 12, replace=False))
    for c in idx:
        lvc = W.uniform_levels(3, int(c), 1, nb, 3)[0]
        assert O.simulate(pl, n, b, lvc, schedule=False)["makespan"] == ms[c], c


def test_build_apart_then_reuse():
    """hesp_dag_build_kept (no platform) followed by reuse launches on two
    platforms equals separate hesp_simulate_batch calls; a failed build keeps
    its status."""
    C, nb = 256, 120
    lvh = W.workload_levels("cfg1", 9000, C)
    lvh[5, 3] = 4  # above max_level: the build fails (HESP_ERR_ARG)
    lv = torch.from_numpy(lvh.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(8, 2048, np.arange(C, dtype=np.int64) * nb)
    ws = hesp.alloc_workspace_kept(8, 2, C)
    nt0 = torch.empty(C, dtype=torch.int64, device="cuda")
    bst, _ = hesp.dag_build_kept(cands, lv, C, 8, 2, ws, ntasks=nt0)
    for key in ("cfg1a", "cfg1b", "cfg2"):
        plat = hesp.Platform(W.PLATFORMS[key])
        ms, st, _ = hesp.simulate_batch_reuse(plat, cands, lv, C, 8, 2, ws)
        ms2, st2, _ = hesp.simulate_batch(plat, cands, lv, C, 8, 2, hesp.alloc_workspace(plat, 8, 2, C))
        torch.cuda.synchronize()
        assert torch.equal(st, st2) and torch.equal(ms, ms2), key
    bst = bst.cpu().numpy()
    assert bst[5] == -1 and (np.delete(bst, 5) == 0).all()


def test_pl_hand_derived_schedule_on_gpu():
    """The hand-derived PL and FCFS schedules of the golden file (3
    processors of two types in one memory, the syrk of a 2 x 2-tile Cholesky
    split once; PL and FCFS differ): the GPU reproduces every processor,
    start and finish of both, from the worked-out values, not from the oracle."""
    import dataclasses
    e = GOLD["n2_b1024_syrk_split_pl_vs_fcfs_p3"]
    spec = dataclasses.replace(W.big_little_platform(), procs=tuple(tuple(p) for p in e["procs"]),
                               exec_overrides=tuple(tuple(x) for x in e["overrides"]))
    lv = np.array([e["levels"]], np.int8)
    for order, want in ((1, e["pl"]), (0, e["fcfs"])):
        plat = hesp.Platform(spec, order=order, select=0)
        d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
        cands = hesp.cands_tensor(e["n"], e["b"], np.zeros(1, np.int64))
        ws = hesp.alloc_workspace(plat, e["n"], 1, 1)
        T = len(want["proc"])
        sched = (torch.zeros(1, dtype=torch.int64, device="cuda"), torch.empty(T, dtype=torch.int16, device="cuda"),
                 torch.empty(T, dtype=torch.int64, device="cuda"), torch.empty(T, dtype=torch.int64, device="cuda"))
        ms, st, _ = hesp.simulate_batch(plat, cands, d_lv, 1, e["n"], 1, ws, schedule=sched)
        torch.cuda.synchronize()
        assert int(st.item()) == 0 and int(ms.item()) == want["makespan"], order
        assert sched[1].cpu().tolist() == want["proc"], order
        assert sched[2].cpu().tolist() == want["start"], order
        assert sched[3].cpu().tolist() == want["finish"], order
