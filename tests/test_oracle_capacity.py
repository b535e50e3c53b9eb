"""Pins of the oracle's finite memory spaces (CPU only).

Sec. 2 describes platforms of finite-size memory spaces; the paper gives no
eviction policy.  The oracle's reading: a bounded accelerator memory can
take a task when the atoms it lacks fit in the free space plus what may be
evicted (atoms the task does not use and no task in flight there still
uses); processors of memories that cannot take the task are skipped;
eviction is least-recently-used (latest finish of a task that used the
atom there, ties to the lower atom); an evicted atom valid nowhere else is
written back to host memory in one message issued at the scheduling time.

Pins: two hand-derived examples (eviction with write-back on a lone GPU; a
GPU too small for two blocks, which sends work to the CPU and changes the
makespan from 73,003 ns to 523,003 ns), capacity above the whole matrix =
the unbounded schedule, capacity below any task = the CPU-only schedule,
and the argument checks.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_05510_b300 import workloads as W

B = 256
ATOM = B * B * 8  # bytes of one 256 x 256 block of doubles (the atom at level 0)


def two_mem_spec(procs):
    """CPU type 0, GPU type 1; task times fixed by overrides (GPU chol 10 us,
    trsm 20 us, syrk 30 us; CPU ten times slower); a message of k atoms takes
    1000 + k ns."""
    ty = {"peak_gflops": 10, "h": 0, "eff_pct": [100, 100, 100, 100]}
    ovr = [(0, 1, B, 10_000), (1, 1, B, 20_000), (2, 1, B, 30_000),
           (0, 0, B, 100_000), (1, 0, B, 200_000), (2, 0, B, 300_000)]
    return {"n_mem": 2, "types": [ty, ty], "procs": procs, "xfer_latency_ns": 1000, "bytes_per_elem": 8,
            "bw_bytes_per_ns": ATOM, "exec_overrides": ovr}


def test_lone_gpu_evicts_and_writes_back():
    """n = 2 tiles, one GPU (memory 1, room for 2 blocks), data in host memory:
    chol(0) fetches A00 (arrives 1,001), ends 11,001; trsm(0,1) fetches A01
    (12,002), ends 32,002; syrk(0,1) needs A11 with A00 and A01 resident:
    A00 (last used until 32,002, not used by syrk) is evicted and, valid
    nowhere else, written back; A11 arrives 33,003, syrk ends 63,003;
    chol(1) finds A11 resident and ends 73,003."""
    spec = two_mem_spec([(1, 1)])
    lv = np.zeros(4, np.int8)
    free = O.simulate(O.make_platform(spec), 2, B, lv)
    cap = O.simulate(O.make_platform(spec, capacity={1: 2 * ATOM}), 2, B, lv)
    assert free["status"] == 0 and cap["status"] == 0
    assert free["makespan"] == cap["makespan"] == 73_003
    assert list(cap["finish"]) == [11_001, 32_002, 63_003, 73_003]
    assert (free["evicted"], free["written_back"]) == (0, 0)
    assert (cap["evicted"], cap["written_back"]) == (1, 1)
    # room for one block only: trsm(0,1) needs two and nothing else can run it
    one = O.simulate(O.make_platform(spec, capacity={1: ATOM}), 2, B, lv)
    assert one["status"] == -2


def test_small_gpu_sends_work_to_the_cpu():
    """CPU (memory 0) + GPU (memory 1, room for one block).  chol(0) on the
    GPU ends 11,001.  trsm(0,1) cannot fit A00 + A01 on the GPU: the CPU runs
    it, fetching A00 back (12,002), and ends 212,002.  syrk(0,1) needs A01
    and A11 on the GPU, where only A00 may go: the CPU runs it, ends 512,002.
    chol(1) fits after evicting A00 (host already has it, so no write-back):
    A11 arrives 513,003, chol ends 523,003 (unbounded: 73,003)."""
    spec = two_mem_spec([(0, 0), (1, 1)])
    lv = np.zeros(4, np.int8)
    free = O.simulate(O.make_platform(spec), 2, B, lv)
    cap = O.simulate(O.make_platform(spec, capacity={1: ATOM}), 2, B, lv)
    assert free["makespan"] == 73_003 and list(free["proc"]) == [1, 1, 1, 1]
    assert cap["status"] == 0 and cap["makespan"] == 523_003
    assert list(cap["proc"]) == [1, 0, 0, 1]
    assert list(cap["finish"]) == [11_001, 212_002, 512_002, 523_003]
    assert (cap["evicted"], cap["written_back"]) == (1, 0)
    # a capacity that is not a whole number of blocks rounds down
    assert O.simulate(O.make_platform(spec, capacity={1: 2 * ATOM - 1}), 2, B, lv)["makespan"] == 523_003


@pytest.mark.parametrize("cache", [0, 1, 2])
@pytest.mark.parametrize("order,select", [(0, 0), (1, 0), (0, 1)])
def test_capacity_above_the_matrix_is_unbounded(cache, order, select):
    spec = W.PLATFORMS["cfg1a"]
    n, b = 8, 2048
    lv = W.workload_levels("cfg1", 40, 6)
    whole = (n * b) ** 2 * spec.bytes_per_elem
    for c in range(lv.shape[0]):
        a = O.simulate(O.make_platform(spec, order, select, cache=cache), n, b, lv[c])
        z = O.simulate(O.make_platform(spec, order, select, cache=cache, capacity={1: whole}), n, b, lv[c])
        assert z["status"] == 0 and z["evicted"] == 0
        assert z["makespan"] == a["makespan"]
        assert np.array_equal(z["proc"], a["proc"]) and np.array_equal(z["finish"], a["finish"])


@pytest.mark.parametrize("select", [0, 1])
def test_capacity_below_any_task_is_the_cpu_only_platform(select):
    """A GPU memory smaller than one atom can take no task: under FCFS every
    task runs on the CPUs exactly as on the same machine without the GPU.
    (Under PL the priorities sum task times over every processor, the GPU
    included, so the two machines order tasks differently.)"""
    n, b = 6, 2048
    lv = np.random.default_rng(4).integers(0, 3, (6, W.base_count(n))).astype(np.int8)
    gpu = O.make_platform(W.cpu_gpu_platform(4, 1), 0, select, capacity={1: 1024})
    cpu = O.make_platform(W.cpu_gpu_platform(4, 0), 0, select)
    for c in range(lv.shape[0]):
        a = O.simulate(gpu, n, b, lv[c])
        z = O.simulate(cpu, n, b, lv[c])
        assert a["status"] == 0 and a["makespan"] == z["makespan"]
        assert np.array_equal(a["proc"], z["proc"]) and np.array_equal(a["start"], z["start"])


def test_capacity_argument_checks():
    spec = W.PLATFORMS["cfg1a"]
    lv = np.zeros(W.base_count(3), np.int8)
    assert O.simulate(O.make_platform(spec, capacity={0: 1 << 30}), 3, 2048, lv)["status"] == -1  # host
    assert O.simulate(O.make_platform(spec, select=2, capacity={1: 1 << 30}), 3, 2048, lv)["status"] == -1
    assert O.simulate(O.make_platform(spec, select=3, capacity={1: 1 << 30}), 3, 2048, lv)["status"] == -1
    assert O.simulate(O.make_platform(spec, capacity={1: -5}), 3, 2048, lv)["status"] == -1
