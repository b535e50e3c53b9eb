"""hesp_simulate_batch_noalloc -- the simulation entry point for callers that
cannot allocate device memory (it uses the library's fixed scratch array
instead of a caller workspace).  Its results must equal those of
hesp_simulate_batch bit for bit (integer nanoseconds), on two calls in a row
that reuse the same array, and sizes beyond the array must be refused.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test."""
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


def _batch(key, first, C):
    w = W.WORKLOADS[key]
    nb = W.base_count(w.n_tiles)
    lv = W.workload_levels(key, first, C)
    levels = torch.from_numpy(lv.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(w.n_tiles, w.b, np.arange(C, dtype=np.int64) * nb)
    return w, lv, levels, cands


def _schedule(w, lv, max_level):
    dag = hesp.Dag(w.n_tiles, w.b, max_level)
    cnt = np.array([dag.count_tasks(r)[0] for r in lv], np.int64)
    off = np.zeros(len(lv) + 1, np.int64)
    off[1:] = np.cumsum(cnt)
    tot = int(off[-1])
    return (torch.from_numpy(off[:-1].copy()).cuda(), torch.empty(tot, dtype=torch.int16, device="cuda"),
            torch.empty(tot, dtype=torch.int64, device="cuda"), torch.empty(tot, dtype=torch.int64, device="cuda"))


@pytest.mark.parametrize("key,plat,max_level", [("cfg1", "cfg1a", 2), ("cfg1", "cfg1b", 2), ("cfg0", "cfg0", 1)])
def test_noalloc_matches_workspace_entry_point_twice(key, plat, max_level):
    p = hesp.Platform(W.PLATFORMS[plat])
    for call, first in enumerate((0, 777)):
        C = 600 if key == "cfg1" else 1024
        w, lv, levels, cands = _batch(key, first if key == "cfg1" else 0, C)
        ws = hesp.alloc_workspace(p, w.n_tiles, max_level, C)
        s_ref = _schedule(w, lv, max_level)
        s_na = _schedule(w, lv, max_level)
        nt_ref = torch.empty(C, dtype=torch.int64, device="cuda")
        nt_na = torch.empty(C, dtype=torch.int64, device="cuda")
        ms_ref, st_ref, _ = hesp.simulate_batch(p, cands, levels, C, w.n_tiles, max_level, ws, ntasks=nt_ref,
                                                schedule=s_ref)
        ms_na, st_na, _ = hesp.simulate_batch_noalloc(p, cands, levels, C, w.n_tiles, max_level, ntasks=nt_na,
                                                      schedule=s_na)
        torch.cuda.synchronize()
        assert (st_ref == 0).all() and (st_na == 0).all(), call
        assert torch.equal(ms_ref, ms_na), call
        assert torch.equal(nt_ref, nt_na), call
        for a, b in zip(s_ref[1:], s_na[1:]):
            assert torch.equal(a, b), call


def test_noalloc_refuses_sizes_beyond_its_array():
    p = hesp.Platform(W.PLATFORMS["cfg4"])
    levels = torch.zeros(16, dtype=torch.int8, device="cuda")
    cands = hesp.cands_tensor(32, 2048, [0])
    with pytest.raises(hesp.HespError) as e:
        hesp.simulate_batch_noalloc(p, cands, levels, 1, 32, 3)
    assert e.value.code == -2  # HESP_ERR_CAPACITY
