"""Host-side arithmetic of bench.py (CPU only): the roofline of the
simulation launch is a per-launch quantity (it does not change when the
number of timed steps does), and the algorithmic operation count per
task-event matches its definition on hand-countable partitions."""
import types

import numpy as np
import pytest

import bench
from paper_1602_05510_b300 import workloads as W


def _props(sms=148):
    return types.SimpleNamespace(multi_processor_count=sms)


def test_roofline_is_per_launch():
    peaks = {"sm_max_mhz": 2032.0}
    a = bench.roofline(3.9, 3.3e9, _props(), peaks)
    b = bench.roofline(2 * 3.9, 2 * 3.3e9, _props(), peaks)  # e.g. two launches timed together
    assert a["frac"] == pytest.approx(b["frac"], rel=1e-12)
    assert a["achieved"] == pytest.approx(a["alg_ops_per_task_event"] * 3.3e9 / 3.9 / 1e12, rel=1e-12)
    assert a["peak"] == pytest.approx(148 * 128 * 2032e6 / 2 / 1e12)
    # the peak follows the device's SM count
    assert bench.roofline(3.9, 3.3e9, _props(160), peaks)["peak"] == pytest.approx(a["peak"] * 160 / 148)


def test_alg_ops_per_event_hand_counts():
    # unsplit 3 x 3 tiles: 3 chol (1 region), 3 trsm (2), 3 syrk (2), 1 gemm (3)
    # = 18 regions over 10 tasks, one atom per region
    lv = np.zeros((1, 10), np.int8)
    assert bench.alg_ops_per_event(lv, 3, 1024, 5, 2) == pytest.approx(4 * 5 + 3 * 18 / 10)
    # one chol split once on 1 tile: chol, trsm, syrk, chol at half size over
    # atoms of half size: regions 1 + 2 + 2 + 1 = 6 atoms over 4 tasks
    assert bench.alg_ops_per_event(np.ones((1, 1), np.int8), 1, 1024, 1, 1) == pytest.approx(4 + 2 * 6 / 4)
    # mixed levels on 2 tiles: the unsplit tasks count 4 atoms per region
    lv = np.array([[1, 0, 0, 0]], np.int8)
    tasks = 4 + 3
    atoms = 6 + 4 * (2 + 2 + 1)
    assert bench.alg_ops_per_event(lv, 2, 1024, 3, 2) == pytest.approx(12 + 3 * atoms / tasks)


def test_workload_constants():
    assert W.base_count(bench.N_TILES) == 5984
    assert bench.N_LEVELS == 4 and bench.N_CAND == 4096
    spec = W.PLATFORMS[bench.PLAT]
    assert len(spec.procs) == 34 and spec.n_mem == 3


def test_reference_arm_line(capsys):
    """bench.py --impl reference: the oracle on one candidate of the default
    workload prints one JSON line with the base contract's keys."""
    import json

    args = types.SimpleNamespace(steps=1, warmup=0, ref_sample=1)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["n_tiles"] == 32 and line["higher_is_better"] is True
