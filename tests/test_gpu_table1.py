"""Table 1 procedure on the GPU (paper_1602_05510_b300.table1: homogeneous
tile-size sweep, then the iterative solver, with hesp_schedule_metrics)
against the oracle's (oracle/metrics.py): the same homogeneous block, the
same heterogeneous partition, and identical integer metrics (makespan, busy
time, task count, summed block size, depth) for several policies; plus the
metrics kernel against the oracle on a batch of random partitions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import metrics as X  # noqa: E402
from paper_1602_05510_b300 import hesp  # noqa: E402
from paper_1602_05510_b300 import table1 as TB  # noqa: E402
from paper_1602_05510_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

KEYS = ("makespan", "busy", "tasks", "sum_block", "depth")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


@pytest.mark.parametrize("key,n,b,L", [("cfg1a", 8, 2048, 2), ("cfg1b", 6, 1024, 2), ("cfg4", 4, 2048, 3)])
def test_metrics_kernel_parity(key, n, b, L):
    spec = W.PLATFORMS[key]
    nb = W.base_count(n)
    C = 16
    lv = np.random.default_rng(n + L).integers(0, L + 1, (C, nb)).astype(np.int8)
    plat = hesp.Platform(spec)
    d_lv = torch.from_numpy(lv.reshape(-1).copy()).cuda()
    cands = hesp.cands_tensor(n, b, np.arange(C, dtype=np.int64) * nb)
    ws = hesp.alloc_workspace(plat, n, L, C)
    dag = hesp.Dag(n, b, L)
    cnt = np.array([dag.count_tasks(lv[c])[0] for c in range(C)], np.int64)
    offs = np.concatenate([[0], np.cumsum(cnt)])
    tot = int(offs[-1])
    sched = (torch.from_numpy(offs[:-1].copy()).cuda(), torch.empty(tot, dtype=torch.int16, device="cuda"),
             torch.empty(tot, dtype=torch.int64, device="cuda"), torch.empty(tot, dtype=torch.int64, device="cuda"))
    ms, st, _ = hesp.simulate_batch(plat, cands, d_lv, C, n, L, ws, schedule=sched)
    busy, nt, sb, dp = (x.cpu().numpy() for x in hesp.schedule_metrics(cands, d_lv, C, schedule=sched))
    _, _, sb2, _ = (x.cpu().numpy() for x in hesp.schedule_metrics(cands, d_lv, C))
    ms = ms.cpu().numpy()
    pl = O.make_platform(spec)
    for c in range(C):
        m = X.metrics(pl, n, b, lv[c])
        assert (ms[c], busy[c], nt[c], sb[c], dp[c]) == tuple(m[k] for k in KEYS), c
        assert sb2[c] == sb[c]


@pytest.mark.parametrize("name,order,select", [TB.POLICIES[0], TB.POLICIES[3], TB.POLICIES[4], TB.POLICIES[7]])
@pytest.mark.parametrize("key,N,sizes", [("cfg1b", 4096, (512, 1024, 2048)), ("cfg0", 4096, (512, 1024, 2048))])
def test_table_row_parity(name, order, select, key, N, sizes):
    spec = W.PLATFORMS[key]
    g = TB.table_row(spec, N, sizes, order, select, rp_seed=3, max_level=2, iterations=8, seed=21)
    o = X.table_row(spec, N, sizes, order, select, 3, 2, 8, 21)
    assert g["homog_block"] == o["homog_block"], name
    assert tuple(g["homog"][k] for k in KEYS) == tuple(o["homog"][k] for k in KEYS)
    assert g["het_levels"].tolist() == o["het_levels"].tolist()
    assert tuple(g["het"][k] for k in KEYS) == tuple(o["het"][k] for k in KEYS)
    assert g["iterations"] == o["iterations"]
    assert g["het"]["makespan"] <= g["homog"]["makespan"]
