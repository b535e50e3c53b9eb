"""Runtime services: CUDA-graph capture/replay of library calls and the
simulator's launch-shape autotuner (results must not depend on the shape)."""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1602_05510_b300 import hesp  # noqa: E402
from paper_1602_05510_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


def test_graph_replay_of_generate_and_simulate():
    C, nb = 2048, 120
    plat = hesp.Platform(W.PLATFORMS["cfg1a"])
    ws = hesp.alloc_workspace(plat, 8, 2, C)
    lv = torch.empty(C * nb, dtype=torch.int8, device="cuda")
    cd = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    ms = torch.empty(C, dtype=torch.int64, device="cuda")
    st = torch.empty(C, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    # direct run first (also sets the kernel attributes outside the capture)
    hesp.generate_candidates(hesp.GEN_UNIFORM, 1, 0, C, 8, 2048, 3, lv, cd, stream=s)
    hesp.simulate_batch(plat, cd, lv, C, 8, 2, ws, makespan=ms, status=st, stream=s)
    s.synchronize()
    ref = ms.clone()
    ms.fill_(-7)
    g = hesp.Graph.capture(s, lambda: (
        hesp.generate_candidates(hesp.GEN_UNIFORM, 1, 0, C, 8, 2048, 3, lv, cd, stream=s),
        hesp.simulate_batch(plat, cd, lv, C, 8, 2, ws, makespan=ms, status=st, stream=s)))
    for _ in range(2):
        ms.fill_(-7)
        torch.cuda.synchronize()
        g.launch(s)
        s.synchronize()
        assert (st == 0).all() and torch.equal(ms, ref)


def test_autotune_picks_a_shape_and_results_do_not_change():
    C = 4096
    plat = hesp.Platform(W.PLATFORMS["cfg1a"])
    ws = hesp.alloc_workspace(plat, 8, 2, C)
    lv = torch.from_numpy(W.workload_levels("cfg1", 0, C).reshape(-1).copy()).cuda()
    cd = hesp.cands_tensor(8, 2048, np.arange(C) * 120)
    ms0, st0, _ = hesp.simulate_batch(plat, cd, lv, C, 8, 2, ws)
    ms0 = ms0.clone()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        (c, b), times = hesp.autotune(plat, cd, lv, C, 8, 2, ws, cache_path=path)
        assert 1 <= c <= 4 and b in (1, 2)
        assert sum(t > 0 for t in times) == 8
        assert hesp.get_tuning(plat) == (c, b)
        for cc in (1, 3):
            for bb in (1, 2):
                hesp.set_tuning(plat, cc, bb)
                ms1, st1, _ = hesp.simulate_batch(plat, cd, lv, C, 8, 2, ws)
                torch.cuda.synchronize()
                assert (st1 == 0).all() and torch.equal(ms1, ms0)
        # the cache answers the second time without timing
        plat2 = hesp.Platform(W.PLATFORMS["cfg1a"])
        (c2, b2), times2 = hesp.autotune(plat2, cd, lv, C, 8, 2, ws, cache_path=path)
        assert (c2, b2) == (c, b) and all(t < 0 for t in times2)


def test_sort_by_size_orders_and_preserves_results():
    from paper_1602_05510_b300 import workloads as W2
    C = 512
    n, b, off, lvh = W2.uneven_candidates(2, 100, C)
    cands = torch.empty(C * 16, dtype=torch.uint8, device="cuda")
    lv = torch.empty(int(off[-1]), dtype=torch.int8, device="cuda")
    used = torch.zeros(1, dtype=torch.int64, device="cuda")
    hesp.generate_uneven(2, 100, C, cands, lv, used)
    sc, perm = hesp.sort_cands_by_size(cands, lv, C)
    plat = hesp.Platform(W2.PLATFORMS["cfg2"])
    ws = hesp.alloc_workspace(plat, 32, 2, C, task_cap=100000)
    nt_s = torch.empty(C, dtype=torch.int64, device="cuda")
    nt_u = torch.empty(C, dtype=torch.int64, device="cuda")
    ms_s, st_s, _ = hesp.simulate_batch(plat, sc, lv, C, 32, 2, ws, ntasks=nt_s, task_cap=100000)
    ms_s = ms_s.clone()
    ms_u, st_u, _ = hesp.simulate_batch(plat, cands, lv, C, 32, 2, ws, ntasks=nt_u, task_cap=100000)
    torch.cuda.synchronize()
    p = perm.cpu().numpy().astype(np.int64)
    assert sorted(p.tolist()) == list(range(C))
    T = nt_s.cpu().numpy()
    assert (np.diff(T // 16) <= 0).all()          # non-increasing in buckets of 16 tasks
    assert (st_s == 0).all() and (st_u == 0).all()
    assert np.array_equal(ms_s.cpu().numpy(), ms_u.cpu().numpy()[p])
