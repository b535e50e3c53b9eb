"""Thin ctypes binding of libhesp.so (C ABI in include/hesp.h).

Argument marshalling only: every step of the simulation and of the surrogate
runs in the library's CUDA kernels.  PyTorch supplies device memory and the
current stream.  There is no CPU fallback: if the library is missing or no
CUDA device is usable, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhesp.so")

HESP_OK = 0
HESP_ERR_ARG, HESP_ERR_CAPACITY, HESP_ERR_UNSUPPORTED = -1, -2, -6
STATUS_NAMES = {0: "HESP_OK", -1: "HESP_ERR_ARG", -2: "HESP_ERR_CAPACITY", -3: "HESP_ERR_CUDA",
                -4: "HESP_ERR_TIMEOUT", -5: "HESP_ERR_STATE", -6: "HESP_ERR_UNSUPPORTED"}
GEN_EXHAUSTIVE, GEN_UNIFORM = 0, 1
MAX_LEVEL, MAX_TILES, MAX_PROCS, MAX_MEMS, MAX_TYPES = 4, 64, 64, 4, 4
MAX_FACTOR = 4  # partition factors k (p = 1/k) of simulate_factors

# Every symbol include/hesp.h declares (checked by the CPU tests).
EXPORTS = (
    "hesp_status_string", "hesp_platform_create", "hesp_platform_set_exec_table", "hesp_platform_exec_ns",
    "hesp_platform_xfer_ns", "hesp_platform_destroy", "hesp_dag_build", "hesp_dag_n_base",
    "hesp_dag_base_tasks", "hesp_dag_count_tasks", "hesp_dag_destroy", "hesp_sim_workspace_size",
    "hesp_simulate_batch", "hesp_simulate_batch_noalloc", "hesp_generate_candidates", "hesp_generate_uneven",
    "hesp_gemm_bf16", "hesp_surrogate_create", "hesp_surrogate_destroy", "hesp_surrogate_shape",
    "hesp_surrogate_set_stats", "hesp_surrogate_get_stats", "hesp_surrogate_fit_stats", "hesp_surrogate_get",
    "hesp_surrogate_set", "hesp_surrogate_grad", "hesp_surrogate_adam", "hesp_surrogate_train",
    "hesp_surrogate_infer", "hesp_surrogate_error", "hesp_select_workspace_size", "hesp_select_topk",
    "hesp_make_cands", "hesp_gather_f32", "hesp_rank_metrics_workspace_size", "hesp_rank_metrics",
    "hesp_generate_mutants", "hesp_gather_rows", "hesp_best_makespan", "hesp_best_candidate", "hesp_graph_begin",
    "hesp_graph_end",
    "hesp_graph_launch", "hesp_graph_destroy", "hesp_platform_set_tuning", "hesp_platform_get_tuning",
    "hesp_sim_autotune", "hesp_sort_cands_workspace_size", "hesp_sort_cands_by_size", "hesp_platform_set_policy",
    "hesp_simulate_critical", "hesp_solver_moves", "hesp_solver_pick", "hesp_schedule_metrics",
    "hesp_sim_workspace_size_factors", "hesp_simulate_factors", "hesp_platform_set_capacity",
    "hesp_solver_moves_range",
    "hesp_sim_workspace_size_kept", "hesp_simulate_batch_keep", "hesp_simulate_batch_reuse",
    "hesp_platform_set_cache", "hesp_surrogate_save", "hesp_surrogate_load", "hesp_platform_set_link",
    "hesp_dag_build_kept",
)
CACHE_WB, CACHE_WT, CACHE_WA = 0, 1, 2
SOLVER_ALL, SOLVER_CP, SOLVER_SHALLOW = 0, 1, 2
PICK_HARD, PICK_SOFT = 0, 1
ORDER_FCFS, ORDER_PL = 0, 1
SELECT_EFT, SELECT_EIT, SELECT_FP, SELECT_RP = 0, 1, 2, 3
NOALLOC_SCRATCH_BYTES = 64 << 20

CAND_DTYPE = np.dtype([("n_tiles", "<i4"), ("b", "<i4"), ("level_offset", "<i8")])


class HespError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed: %s (%d)" % (what, STATUS_NAMES.get(code, "?"), code))
        self.code = code


class _PType(ctypes.Structure):
    _fields_ = [("peak_gflops", ctypes.c_int64), ("h", ctypes.c_int64), ("eff_pct", ctypes.c_int32 * 4)]


class _Proc(ctypes.Structure):
    _fields_ = [("memory", ctypes.c_int32), ("type", ctypes.c_int32)]


class _PlatDesc(ctypes.Structure):
    _fields_ = [("n_mem", ctypes.c_int32), ("n_types", ctypes.c_int32), ("types", ctypes.POINTER(_PType)),
                ("n_procs", ctypes.c_int32), ("procs", ctypes.POINTER(_Proc)),
                ("xfer_latency_ns", ctypes.c_int64), ("bytes_per_elem", ctypes.c_int64),
                ("bw_bytes_per_ns", ctypes.c_int64)]


_lib = None


def lib():
    """Load libhesp.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhesp.so not built: run `python -m paper_1602_05510_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        i32, i64, u64, vp, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t
        L.hesp_status_string.restype = ctypes.c_char_p
        L.hesp_status_string.argtypes = [ctypes.c_int]
        L.hesp_platform_create.argtypes = [ctypes.POINTER(_PlatDesc), ctypes.POINTER(vp)]
        L.hesp_platform_set_exec_table.argtypes = [vp, i32, i32, i64, i64]
        L.hesp_platform_exec_ns.argtypes = [vp, i32, i32, i64, ctypes.POINTER(i64)]
        L.hesp_platform_xfer_ns.argtypes = [vp, i64, ctypes.POINTER(i64)]
        L.hesp_platform_destroy.argtypes = [vp]
        L.hesp_platform_destroy.restype = None
        L.hesp_dag_build.argtypes = [i32, i32, i32, ctypes.POINTER(vp)]
        L.hesp_dag_n_base.argtypes = [vp]
        L.hesp_dag_n_base.restype = i64
        L.hesp_dag_base_tasks.argtypes = [vp, vp, vp, vp, vp]
        L.hesp_dag_count_tasks.argtypes = [vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.hesp_dag_destroy.argtypes = [vp]
        L.hesp_dag_destroy.restype = None
        L.hesp_sim_workspace_size.argtypes = [vp, i32, i32, i64, i64, ctypes.POINTER(sz)]
        L.hesp_simulate_batch.argtypes = [vp, vp, vp, i64, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.hesp_simulate_batch_noalloc.argtypes = [vp, vp, vp, i64, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.hesp_simulate_critical.argtypes = [vp, vp, vp, i64, i32, i32, i64, vp, vp, vp, vp, sz, vp]
        L.hesp_platform_set_capacity.argtypes = [vp, i32, i64]
        L.hesp_sim_workspace_size_factors.argtypes = [vp, i32, i32, i64, i64, ctypes.POINTER(sz)]
        L.hesp_simulate_factors.argtypes = [vp, vp, vp, i64, i32, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                            sz, vp]
        L.hesp_solver_moves_range.argtypes = [vp, i32, i32, i32, i32, vp, vp, vp, vp, vp]
        L.hesp_sim_workspace_size_kept.argtypes = [i32, i32, i64, i64, ctypes.POINTER(sz)]
        L.hesp_simulate_batch_keep.argtypes = [vp, vp, vp, i64, i32, i32, i64, vp, vp, vp, vp, sz, vp]
        L.hesp_dag_build_kept.argtypes = [vp, vp, i64, i32, i32, i64, vp, vp, vp, sz, vp]
        L.hesp_simulate_batch_reuse.argtypes = [vp, vp, vp, i64, i32, i32, i64, vp, vp, vp, vp, sz, vp]
        L.hesp_solver_moves.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, vp]
        L.hesp_solver_pick.argtypes = [vp, vp, vp, vp, i32, u64, i64, vp, vp, vp, vp]
        L.hesp_schedule_metrics.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.hesp_gemm_bf16.argtypes = [i32, i32, i32, vp, i64, vp, i64, i32, vp, i64, vp, vp, i64, vp, i64, vp, i64,
                                     vp, vp]
        f32, f64 = ctypes.c_float, ctypes.c_double
        L.hesp_surrogate_create.argtypes = [i32, i32, i32, i32, u64, ctypes.POINTER(vp)]
        L.hesp_surrogate_save.argtypes = [vp, ctypes.c_char_p]
        L.hesp_surrogate_load.argtypes = [ctypes.c_char_p, vp]
        L.hesp_surrogate_destroy.argtypes = [vp]
        L.hesp_surrogate_destroy.restype = None
        L.hesp_surrogate_shape.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]
        L.hesp_surrogate_set_stats.argtypes = [vp, f64, f64]
        L.hesp_surrogate_get_stats.argtypes = [vp, ctypes.POINTER(f64), ctypes.POINTER(f64), ctypes.POINTER(i64)]
        L.hesp_surrogate_fit_stats.argtypes = [vp, vp, i64, vp]
        L.hesp_surrogate_get.argtypes = [vp, i32, vp, i64]
        L.hesp_surrogate_set.argtypes = [vp, i32, vp, i64]
        L.hesp_surrogate_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.hesp_surrogate_adam.argtypes = [vp, f32, vp]
        L.hesp_surrogate_train.argtypes = [vp, vp, vp, i64, i32, i32, f32, u64, vp, vp]
        L.hesp_surrogate_infer.argtypes = [vp, vp, i64, vp, vp]
        L.hesp_surrogate_error.argtypes = [vp, ctypes.POINTER(i32)]
        L.hesp_select_workspace_size.argtypes = [i64, ctypes.POINTER(sz)]
        L.hesp_select_topk.argtypes = [vp, i64, i64, vp, vp, sz, vp]
        L.hesp_make_cands.argtypes = [vp, i64, i32, i32, vp, vp]
        L.hesp_gather_f32.argtypes = [vp, vp, i64, vp, vp]
        L.hesp_rank_metrics_workspace_size.argtypes = [i64, ctypes.POINTER(sz)]
        L.hesp_rank_metrics.argtypes = [vp, vp, i64, f64, f64, vp, sz, ctypes.POINTER(f64), vp]
        L.hesp_graph_begin.argtypes = [vp]
        L.hesp_graph_end.argtypes = [vp, ctypes.POINTER(vp)]
        L.hesp_graph_launch.argtypes = [vp, vp]
        L.hesp_graph_destroy.argtypes = [vp]
        L.hesp_graph_destroy.restype = None
        L.hesp_platform_set_tuning.argtypes = [vp, i32, i32]
        L.hesp_platform_get_tuning.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.hesp_sim_autotune.argtypes = [vp, vp, vp, i64, i32, i32, i64, vp, vp, vp, sz, ctypes.c_char_p,
                                        ctypes.POINTER(i32), ctypes.POINTER(i32), vp, vp]
        L.hesp_sort_cands_workspace_size.argtypes = [i64, ctypes.POINTER(sz)]
        L.hesp_sort_cands_by_size.argtypes = [vp, vp, i64, vp, vp, vp, sz, vp]
        L.hesp_platform_set_policy.argtypes = [vp, i32, i32, u64]
        L.hesp_platform_set_cache.argtypes = [vp, i32]
        L.hesp_platform_set_link.argtypes = [vp, i32, i32, i64, i64]
        L.hesp_best_makespan.argtypes = [vp, vp, vp, i64, vp, vp]
        L.hesp_best_candidate.argtypes = [vp, vp, i64, i64, vp, vp]
        L.hesp_gather_rows.argtypes = [vp, vp, i64, i64, vp, vp]
        L.hesp_generate_mutants.argtypes = [vp, i32, i32, i32, ctypes.c_double, u64, i64, i64, vp, vp]
        L.hesp_generate_candidates.argtypes = [i32, u64, i64, i64, i32, i32, i32, vp, vp, vp]
        L.hesp_generate_uneven.argtypes = [u64, i64, i64, vp, vp, i64, vp, vp]
        _lib = L
    return _lib


def check(rc, what):
    if rc != HESP_OK:
        raise HespError(rc, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Platform:
    """A simulated platform (hesp_platform handle) built from a
    ``workloads.PlatformSpec``, with its task order, processor selection,
    R-P seed, caching policy, optional per-link costs {(src, dst):
    (latency_ns, bytes_per_ns)} and optional finite memories {mem: bytes}."""

    def __init__(self, spec, order=0, select=0, rp_seed=0, cache=0, links=None, capacity=None):
        self.spec = spec
        L = lib()
        types = (_PType * len(spec.types))()
        for i, t in enumerate(spec.types):
            types[i].peak_gflops, types[i].h = t.peak_gflops, t.h
            for o in range(4):
                types[i].eff_pct[o] = t.eff_pct[o]
        procs = (_Proc * len(spec.procs))()
        for i, (m, ty) in enumerate(spec.procs):
            procs[i].memory, procs[i].type = m, ty
        d = _PlatDesc(spec.n_mem, len(spec.types), types, len(spec.procs), procs, spec.xfer_latency_ns,
                      spec.bytes_per_elem, spec.bw_bytes_per_ns)
        h = ctypes.c_void_p()
        check(L.hesp_platform_create(ctypes.byref(d), ctypes.byref(h)), "hesp_platform_create")
        self.h = h
        for (op, ty, bs, ns) in getattr(spec, "exec_overrides", ()):
            check(L.hesp_platform_set_exec_table(h, op, ty, bs, ns), "hesp_platform_set_exec_table")
        check(L.hesp_platform_set_policy(h, order, select, rp_seed & ((1 << 64) - 1)), "hesp_platform_set_policy")
        check(L.hesp_platform_set_cache(h, cache), "hesp_platform_set_cache")
        for (s_, d_), (lat, bw) in sorted((links or {}).items()):
            check(L.hesp_platform_set_link(h, s_, d_, lat, bw), "hesp_platform_set_link")
        for m, nbytes in sorted((capacity or {}).items()):
            check(L.hesp_platform_set_capacity(h, m, nbytes), "hesp_platform_set_capacity")

    @property
    def n_mem(self):
        return self.spec.n_mem

    def exec_ns(self, op, ptype, block):
        v = ctypes.c_int64()
        check(lib().hesp_platform_exec_ns(self.h, op, ptype, block, ctypes.byref(v)), "hesp_platform_exec_ns")
        return v.value

    def xfer_ns(self, elems):
        v = ctypes.c_int64()
        check(lib().hesp_platform_xfer_ns(self.h, elems, ctypes.byref(v)), "hesp_platform_xfer_ns")
        return v.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hesp_platform_destroy(self.h)
            self.h = None


class Dag:
    """Base task list of an n x n tiled Cholesky (hesp_dag handle)."""

    def __init__(self, n_tiles, b, max_level):
        h = ctypes.c_void_p()
        check(lib().hesp_dag_build(n_tiles, b, max_level, ctypes.byref(h)), "hesp_dag_build")
        self.h = h
        self.n_tiles, self.b, self.max_level = n_tiles, b, max_level
        self.n_base = int(lib().hesp_dag_n_base(h))

    def base_tasks(self):
        out = [np.zeros(self.n_base, np.int32) for _ in range(4)]
        check(lib().hesp_dag_base_tasks(self.h, *[o.ctypes.data for o in out]), "hesp_dag_base_tasks")
        return out

    def count_tasks(self, levels):
        lv = np.ascontiguousarray(levels, np.int8)
        t = ctypes.c_int64()
        f = ctypes.c_int64()
        check(lib().hesp_dag_count_tasks(self.h, lv.ctypes.data, ctypes.byref(t), ctypes.byref(f)),
              "hesp_dag_count_tasks")
        return t.value, f.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hesp_dag_destroy(self.h)
            self.h = None


def cands_tensor(n_tiles, b, offsets, device="cuda"):
    """hesp_cand[] as a byte tensor on the device."""
    import torch
    offsets = np.asarray(offsets, np.int64)
    a = np.zeros(len(offsets), CAND_DTYPE)
    a["n_tiles"] = n_tiles
    a["b"] = b
    a["level_offset"] = offsets
    return torch.from_numpy(a.view(np.uint8).copy()).to(device)


def workspace_bytes(platform: Platform, max_tiles, max_level, n_cand, task_cap=0):
    v = ctypes.c_size_t()
    check(lib().hesp_sim_workspace_size(platform.h, max_tiles, max_level, task_cap, n_cand, ctypes.byref(v)),
          "hesp_sim_workspace_size")
    return v.value


def alloc_workspace(platform: Platform, max_tiles, max_level, n_cand, task_cap=0, max_bytes=None):
    """Workspace for up to n_cand concurrent candidates (fewer if max_bytes
    would be exceeded)."""
    import torch
    nbytes = workspace_bytes(platform, max_tiles, max_level, n_cand, task_cap)
    if max_bytes is not None and nbytes > max_bytes:
        one = workspace_bytes(platform, max_tiles, max_level, 1, task_cap)
        slot = max(1, workspace_bytes(platform, max_tiles, max_level, 2, task_cap) - one)
        nbytes = max(one, one + (max_bytes - one) // slot * slot)
    return torch.empty(nbytes, dtype=torch.uint8, device="cuda")


def simulate_batch(platform: Platform, cands, levels, n_cand, max_tiles, max_level, workspace,
                   makespan=None, status=None, ntasks=None, schedule=None, stream=None, task_cap=0):
    """Launch hesp_simulate_batch on the current stream.  `cands` is a byte
    tensor of hesp_cand, `levels` an int8 device tensor.  `schedule` is None
    or (offsets int64, proc int16, start int64, finish int64) device tensors.
    Returns (makespan, status, ntasks) device tensors."""
    import torch
    dev = levels.device
    if makespan is None:
        makespan = torch.empty(n_cand, dtype=torch.int64, device=dev)
    if status is None:
        status = torch.empty(n_cand, dtype=torch.int32, device=dev)
    so = sp = ss = sf = None
    if schedule is not None:
        so, sp, ss, sf = schedule
    check(lib().hesp_simulate_batch(platform.h, _ptr(cands), _ptr(levels), n_cand, max_tiles, max_level, task_cap,
                                    _ptr(makespan), _ptr(status), _ptr(ntasks), _ptr(so), _ptr(sp), _ptr(ss),
                                    _ptr(sf), _ptr(workspace), workspace.numel(), _stream(stream)),
          "hesp_simulate_batch")
    return makespan, status, ntasks


def alloc_workspace_factors(platform: Platform, max_tiles, max_factor, n_cand, task_cap=0):
    """Workspace of simulate_factors for up to n_cand concurrent candidates."""
    import torch
    n = ctypes.c_size_t()
    check(lib().hesp_sim_workspace_size_factors(platform.h, max_tiles, max_factor, task_cap, n_cand, ctypes.byref(n)),
          "hesp_sim_workspace_size_factors")
    return torch.empty(n.value, dtype=torch.uint8, device="cuda")


def simulate_factors(platform: Platform, cands, factors, n_cand, max_tiles, max_factor, b, workspace,
                     makespan=None, status=None, ntasks=None, schedule=None, stream=None, task_cap=0, crit=None):
    """hesp_simulate_factors: one partition factor k (p = 1/k) per base task,
    every candidate of block size b.  Arguments and results as
    simulate_batch, with `factors` (int8 device tensor) in place of levels;
    `crit` (int8 device tensor like factors, optional) receives the
    critical-path flags per base task."""
    import torch
    dev = factors.device
    if makespan is None:
        makespan = torch.empty(n_cand, dtype=torch.int64, device=dev)
    if status is None:
        status = torch.empty(n_cand, dtype=torch.int32, device=dev)
    so = sp = ss = sf = None
    if schedule is not None:
        so, sp, ss, sf = schedule
    check(lib().hesp_simulate_factors(platform.h, _ptr(cands), _ptr(factors), n_cand, max_tiles, max_factor, b,
                                      task_cap, _ptr(makespan), _ptr(status), _ptr(ntasks), _ptr(so), _ptr(sp),
                                      _ptr(ss), _ptr(sf), _ptr(crit), _ptr(workspace), workspace.numel(),
                                      _stream(stream)),
          "hesp_simulate_factors")
    return makespan, status, ntasks


def simulate_batch_noalloc(platform: Platform, cands, levels, n_cand, max_tiles, max_level, makespan=None,
                           status=None, ntasks=None, schedule=None, stream=None):
    """hesp_simulate_batch_noalloc: same results as simulate_batch, with the
    library's fixed device scratch array instead of a workspace (for callers
    that cannot allocate device memory).  Calls that overlap on the GPU race
    on that array."""
    import torch
    dev = levels.device
    if makespan is None:
        makespan = torch.empty(n_cand, dtype=torch.int64, device=dev)
    if status is None:
        status = torch.empty(n_cand, dtype=torch.int32, device=dev)
    so = sp = ss = sf = None
    if schedule is not None:
        so, sp, ss, sf = schedule
    check(lib().hesp_simulate_batch_noalloc(platform.h, _ptr(cands), _ptr(levels), n_cand, max_tiles, max_level,
                                            _ptr(makespan), _ptr(status), _ptr(ntasks), _ptr(so), _ptr(sp),
                                            _ptr(ss), _ptr(sf), _stream(stream)),
          "hesp_simulate_batch_noalloc")
    return makespan, status, ntasks


def alloc_workspace_kept(max_tiles, max_level, n_cand, task_cap=0):
    """Workspace of one arena per candidate, for simulate_batch_keep / _reuse."""
    import torch
    n = ctypes.c_size_t()
    check(lib().hesp_sim_workspace_size_kept(max_tiles, max_level, task_cap, n_cand, ctypes.byref(n)),
          "hesp_sim_workspace_size_kept")
    return torch.empty(n.value, dtype=torch.uint8, device="cuda")


def _simulate_kept(fn, name, platform, cands, levels, n_cand, max_tiles, max_level, workspace, makespan, status,
                   ntasks, stream, task_cap):
    import torch
    dev = levels.device
    if makespan is None:
        makespan = torch.empty(n_cand, dtype=torch.int64, device=dev)
    if status is None:
        status = torch.empty(n_cand, dtype=torch.int32, device=dev)
    check(fn(platform.h, _ptr(cands), _ptr(levels), n_cand, max_tiles, max_level, task_cap, _ptr(makespan),
             _ptr(status), _ptr(ntasks), _ptr(workspace), workspace.numel(), _stream(stream)), name)
    return makespan, status, ntasks


def dag_build_kept(cands, levels, n_cand, max_tiles, max_level, workspace, status=None, ntasks=None, stream=None,
                   task_cap=0):
    """hesp_dag_build_kept: build and keep every candidate's DAG (no simulation)."""
    import torch
    if status is None:
        status = torch.empty(n_cand, dtype=torch.int32, device=levels.device)
    check(lib().hesp_dag_build_kept(_ptr(cands), _ptr(levels), n_cand, max_tiles, max_level, task_cap, _ptr(status),
                                    _ptr(ntasks), _ptr(workspace), workspace.numel(), _stream(stream)),
          "hesp_dag_build_kept")
    return status, ntasks


def simulate_batch_keep(platform: Platform, cands, levels, n_cand, max_tiles, max_level, workspace, makespan=None,
                        status=None, ntasks=None, stream=None, task_cap=0):
    """hesp_simulate_batch_keep: simulate and keep each candidate's DAG."""
    return _simulate_kept(lib().hesp_simulate_batch_keep, "hesp_simulate_batch_keep", platform, cands, levels,
                          n_cand, max_tiles, max_level, workspace, makespan, status, ntasks, stream, task_cap)


def simulate_batch_reuse(platform: Platform, cands, levels, n_cand, max_tiles, max_level, workspace, makespan=None,
                         status=None, ntasks=None, stream=None, task_cap=0):
    """hesp_simulate_batch_reuse: simulate the kept DAGs on another platform."""
    return _simulate_kept(lib().hesp_simulate_batch_reuse, "hesp_simulate_batch_reuse", platform, cands, levels,
                          n_cand, max_tiles, max_level, workspace, makespan, status, ntasks, stream, task_cap)


def simulate_critical(platform: Platform, cands, levels, n_cand, max_tiles, max_level, workspace, crit,
                      makespan=None, status=None, stream=None, task_cap=0):
    """hesp_simulate_critical: makespans plus, per base task, a critical-path
    flag written to `crit` (int8, laid out like `levels`)."""
    import torch
    dev = levels.device
    if makespan is None:
        makespan = torch.empty(n_cand, dtype=torch.int64, device=dev)
    if status is None:
        status = torch.empty(n_cand, dtype=torch.int32, device=dev)
    check(lib().hesp_simulate_critical(platform.h, _ptr(cands), _ptr(levels), n_cand, max_tiles, max_level, task_cap,
                                       _ptr(makespan), _ptr(status), _ptr(crit), _ptr(workspace), workspace.numel(),
                                       _stream(stream)), "hesp_simulate_critical")
    return makespan, status


def schedule_metrics(cands, levels, n_cand, schedule=None, stream=None):
    """hesp_schedule_metrics: (busy, ntasks, sum_block, depth) device tensors
    per candidate; `schedule` = the (offsets, proc, start, finish) tensors
    given to simulate_batch, or None (busy is then -1)."""
    import torch
    dev = levels.device
    busy = torch.empty(n_cand, dtype=torch.int64, device=dev)
    nt = torch.empty(n_cand, dtype=torch.int64, device=dev)
    sb = torch.empty(n_cand, dtype=torch.int64, device=dev)
    dp = torch.empty(n_cand, dtype=torch.int32, device=dev)
    so = ss = sf = None
    if schedule is not None:
        so, _, ss, sf = schedule
    check(lib().hesp_schedule_metrics(_ptr(cands), _ptr(levels), n_cand, _ptr(so), _ptr(ss), _ptr(sf), _ptr(busy),
                                      _ptr(nt), _ptr(sb), _ptr(dp), _stream(stream)), "hesp_schedule_metrics")
    return busy, nt, sb, dp


def solver_moves(levels, n_base, n_levels, mode, crit, moves, count, rows=None, stream=None):
    """hesp_solver_moves: candidate moves of the partition `levels`."""
    check(lib().hesp_solver_moves(_ptr(levels), n_base, n_levels, mode, _ptr(crit), _ptr(moves), _ptr(count),
                                  _ptr(rows), _stream(stream)), "hesp_solver_moves")


def solver_moves_range(values, n_base, lo, hi, mode, crit, moves, count, rows=None, stream=None):
    """hesp_solver_moves_range: candidate moves of a partition whose values
    lie in [lo, hi] (partition factors: lo = 1, hi = max_factor)."""
    check(lib().hesp_solver_moves_range(_ptr(values), n_base, lo, hi, mode, _ptr(crit), _ptr(moves), _ptr(count),
                                        _ptr(rows), _stream(stream)), "hesp_solver_moves_range")


def solver_pick(makespan, status, moves, count, pick, seed, iteration, cur_makespan, levels, chosen, stream=None):
    """hesp_solver_pick: score, pick and apply one move (in place)."""
    check(lib().hesp_solver_pick(_ptr(makespan), _ptr(status), _ptr(moves), _ptr(count), pick,
                                 seed & ((1 << 64) - 1), iteration, _ptr(cur_makespan), _ptr(levels), _ptr(chosen),
                                 _stream(stream)), "hesp_solver_pick")


def generate_candidates(kind, seed, first, n_cand, n_tiles, b, n_levels, levels, cands=None, stream=None):
    check(lib().hesp_generate_candidates(kind, seed, first, n_cand, n_tiles, b, n_levels, _ptr(cands),
                                         _ptr(levels), _stream(stream)), "hesp_generate_candidates")


def generate_mutants(parents, n_parents, n_base, n_levels, p_mut, seed, first, n, levels, stream=None):
    check(lib().hesp_generate_mutants(_ptr(parents), n_parents, n_base, n_levels, p_mut, seed, first, n,
                                      _ptr(levels), _stream(stream)), "hesp_generate_mutants")


def generate_uneven(seed, first, n_cand, cands, levels, levels_used, stream=None):
    check(lib().hesp_generate_uneven(seed, first, n_cand, _ptr(cands), _ptr(levels), levels.numel(),
                                     _ptr(levels_used), _stream(stream)), "hesp_generate_uneven")


GEMM_F32, GEMM_BIAS_RELU, GEMM_MASK = 0, 1, 2


def gemm_bf16(A, B, epilogue=GEMM_F32, C=None, bias=None, out=None, out_t=None, mask=None, err=None, K=None,
              stream=None):
    """hesp_gemm_bf16: C[M, N] = A[M, K] B[N, K]^T on the tensor cores.
    A, B: bf16 row-major device tensors (K columns used, a multiple of 64).
    epilogue 0: fp32 C; 1: bf16 out = relu(acc + bias) (+ transposed out_t);
    2: bf16 out = acc where mask > 0 else 0 (+ out_t)."""
    M, N = A.shape[0], B.shape[0]
    K = A.shape[1] if K is None else K
    check(lib().hesp_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), epilogue, _ptr(C),
                               C.stride(0) if C is not None else 0, _ptr(bias), _ptr(out),
                               out.stride(0) if out is not None else 0, _ptr(out_t),
                               out_t.stride(0) if out_t is not None else 0, _ptr(mask),
                               mask.stride(0) if mask is not None else 0, _ptr(err), _stream(stream)),
          "hesp_gemm_bf16")


class Surrogate:
    """The MLP surrogate (hesp_surrogate handle): n_base * n_levels one-hot
    inputs -> hidden -> hidden -> 1, bf16 tensor-core kernels, FP32 masters."""

    PARTS = ("W1", "b1", "W2", "b2", "w3", "b3")

    def __init__(self, n_base, n_levels, hidden=512, max_batch=4096, seed=0, _handle=None):
        h = ctypes.c_void_p()
        if _handle is None:
            check(lib().hesp_surrogate_create(n_base, n_levels, hidden, max_batch, seed, ctypes.byref(h)),
                  "hesp_surrogate_create")
        else:
            h = _handle
        self.h = h
        F, Fp, H = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        check(lib().hesp_surrogate_shape(h, ctypes.byref(F), ctypes.byref(Fp), ctypes.byref(H)),
              "hesp_surrogate_shape")
        self.n_base, self.n_levels, self.F, self.Fp, self.H = n_base, n_levels, F.value, Fp.value, H.value
        self.max_batch = max_batch
        self.sizes = (self.H * self.Fp, self.H, self.H * self.H, self.H, self.H, 1)
        self.shapes = ((self.H, self.Fp), (self.H,), (self.H, self.H), (self.H,), (self.H,), (1,))

    def save(self, path):
        """hesp_surrogate_save: parameters, Adam state and statistics to a file."""
        check(lib().hesp_surrogate_save(self.h, os.fsencode(path)), "hesp_surrogate_save")

    @classmethod
    def load(cls, path):
        """hesp_surrogate_load: a new surrogate from a saved file."""
        h = ctypes.c_void_p()
        check(lib().hesp_surrogate_load(os.fsencode(path), ctypes.byref(h)), "hesp_surrogate_load")
        import struct
        with open(path, "rb") as f:
            n_base, n_levels, H, max_batch = struct.unpack("<4i", f.read(24)[8:24])
        return cls(n_base, n_levels, H, max_batch, _handle=h)

    def _flat(self, parts):
        return np.concatenate([np.asarray(parts[k], np.float32).reshape(-1) for k in self.PARTS])

    def _split(self, flat):
        out, o = {}, 0
        for k, n, sh in zip(self.PARTS, self.sizes, self.shapes):
            out[k] = flat[o:o + n].reshape(sh)
            o += n
        return out

    def get(self, which=0):
        """which: 0 parameters, 1 gradients, 2 Adam first moments, 3 second moments."""
        flat = np.zeros(sum(self.sizes), np.float32)
        check(lib().hesp_surrogate_get(self.h, which, flat.ctypes.data, flat.size), "hesp_surrogate_get")
        return self._split(flat)

    def set(self, parts, which=0):
        flat = np.ascontiguousarray(self._flat(parts))
        check(lib().hesp_surrogate_set(self.h, which, flat.ctypes.data, flat.size), "hesp_surrogate_set")

    def set_stats(self, mu, sigma):
        check(lib().hesp_surrogate_set_stats(self.h, mu, sigma), "hesp_surrogate_set_stats")

    def stats(self):
        mu, sg, st = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        check(lib().hesp_surrogate_get_stats(self.h, ctypes.byref(mu), ctypes.byref(sg), ctypes.byref(st)),
              "hesp_surrogate_get_stats")
        return mu.value, sg.value, st.value

    def fit_stats(self, makespan, stream=None):
        check(lib().hesp_surrogate_fit_stats(self.h, _ptr(makespan), makespan.numel(), _stream(stream)),
              "hesp_surrogate_fit_stats")

    def grad(self, levels, makespan, B, pred=None, loss=None, stream=None):
        check(lib().hesp_surrogate_grad(self.h, _ptr(levels), _ptr(makespan), B, _ptr(pred), _ptr(loss),
                                        _stream(stream)), "hesp_surrogate_grad")

    def adam(self, lr=1e-3, stream=None):
        check(lib().hesp_surrogate_adam(self.h, lr, _stream(stream)), "hesp_surrogate_adam")

    def train(self, levels, makespan, n_samples, batch, n_steps, lr=1e-3, seed=0, loss=None, stream=None):
        check(lib().hesp_surrogate_train(self.h, _ptr(levels), _ptr(makespan), n_samples, batch, n_steps, lr, seed,
                                         _ptr(loss), _stream(stream)), "hesp_surrogate_train")

    def infer(self, levels, n, pred, stream=None):
        check(lib().hesp_surrogate_infer(self.h, _ptr(levels), n, _ptr(pred), _stream(stream)),
              "hesp_surrogate_infer")

    def error_flag(self):
        e = ctypes.c_int32()
        check(lib().hesp_surrogate_error(self.h, ctypes.byref(e)), "hesp_surrogate_error")
        return e.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hesp_surrogate_destroy(self.h)
            self.h = None


def select_topk(keys, k, idx=None, stream=None):
    """Indices (ascending) of the k smallest keys (ties to the lowest index)."""
    import torch
    n = keys.numel()
    sz = ctypes.c_size_t()
    check(lib().hesp_select_workspace_size(n, ctypes.byref(sz)), "hesp_select_workspace_size")
    ws = torch.empty(sz.value, dtype=torch.uint8, device=keys.device)
    if idx is None:
        idx = torch.empty(k, dtype=torch.int64, device=keys.device)
    check(lib().hesp_select_topk(_ptr(keys), n, k, _ptr(idx), _ptr(ws), sz.value, _stream(stream)),
          "hesp_select_topk")
    return idx


def make_cands(idx, n_tiles, b, cands=None, stream=None):
    import torch
    k = idx.numel()
    if cands is None:
        cands = torch.empty(k * 16, dtype=torch.uint8, device=idx.device)
    check(lib().hesp_make_cands(_ptr(idx), k, n_tiles, b, _ptr(cands), _stream(stream)), "hesp_make_cands")
    return cands


def gather_f32(src, idx, dst=None, stream=None):
    import torch
    if dst is None:
        dst = torch.empty(idx.numel(), dtype=torch.float32, device=src.device)
    check(lib().hesp_gather_f32(_ptr(src), _ptr(idx), idx.numel(), _ptr(dst), _stream(stream)), "hesp_gather_f32")
    return dst


def rank_metrics(pred, makespan, mu, sigma, stream=None):
    """(mean relative makespan error, Spearman rank correlation) of the
    surrogate's predictions against exact makespans."""
    import torch
    k = pred.numel()
    sz = ctypes.c_size_t()
    check(lib().hesp_rank_metrics_workspace_size(k, ctypes.byref(sz)), "hesp_rank_metrics_workspace_size")
    ws = torch.empty(sz.value, dtype=torch.uint8, device=pred.device)
    out = (ctypes.c_double * 2)()
    check(lib().hesp_rank_metrics(_ptr(pred), _ptr(makespan), k, mu, sigma, _ptr(ws), sz.value, out,
                                  _stream(stream)), "hesp_rank_metrics")
    return out[0], out[1]


def gather_rows(src, idx, width, dst=None, stream=None):
    """dst[i, :] = src[idx[i], :] for int8 rows (device tensors)."""
    import torch
    k = idx.numel()
    if dst is None:
        dst = torch.empty(k * width, dtype=torch.int8, device=src.device)
    check(lib().hesp_gather_rows(_ptr(src), _ptr(idx), k, width, _ptr(dst), _stream(stream)), "hesp_gather_rows")
    return dst


def best_makespan(makespan, status, ntasks=None, out=None, stream=None):
    """Device int64 [2]: smallest makespan among successful candidates, and
    their task count."""
    import torch
    if out is None:
        out = torch.empty(2, dtype=torch.int64, device=makespan.device)
    check(lib().hesp_best_makespan(_ptr(makespan), _ptr(status), _ptr(ntasks), makespan.numel(), _ptr(out),
                                   _stream(stream)), "hesp_best_makespan")
    return out


def best_candidate(makespan, status, first_index=0, out=None, stream=None):
    """Device int64 [2]: the least makespan among successful candidates and
    first_index + the lowest index holding it (INT64_MAX, -1 if none)."""
    import torch
    if out is None:
        out = torch.empty(2, dtype=torch.int64, device=makespan.device)
    check(lib().hesp_best_candidate(_ptr(makespan), _ptr(status), makespan.numel(), first_index, _ptr(out),
                                    _stream(stream)), "hesp_best_candidate")
    return out


class Graph:
    """A CUDA graph of hesp_* calls captured on a (non-default) stream:

        g = Graph.capture(stream, lambda: ...calls with stream=stream...)
        g.launch(stream)
    """

    def __init__(self, h):
        self.h = h

    @classmethod
    def capture(cls, stream, fn):
        check(lib().hesp_graph_begin(ctypes.c_void_p(stream.cuda_stream)), "hesp_graph_begin")
        try:
            fn()
        finally:
            h = ctypes.c_void_p()
            rc = lib().hesp_graph_end(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        check(rc, "hesp_graph_end")
        return cls(h)

    def launch(self, stream):
        check(lib().hesp_graph_launch(self.h, ctypes.c_void_p(stream.cuda_stream)), "hesp_graph_launch")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hesp_graph_destroy(self.h)
            self.h = None


def set_tuning(platform, ctas_per_sm=0, bitmap_place=0):
    check(lib().hesp_platform_set_tuning(platform.h, ctas_per_sm, bitmap_place), "hesp_platform_set_tuning")


def get_tuning(platform):
    c, b = ctypes.c_int32(), ctypes.c_int32()
    check(lib().hesp_platform_get_tuning(platform.h, ctypes.byref(c), ctypes.byref(b)), "hesp_platform_get_tuning")
    return c.value, b.value


def autotune(platform, cands, levels, n_sample, max_tiles, max_level, workspace, task_cap=0, cache_path=None,
             stream=None):
    """Returns ((ctas_per_sm, bitmap_place), [ms per shape])."""
    import torch
    ms = torch.empty(n_sample, dtype=torch.int64, device=levels.device)
    st = torch.empty(n_sample, dtype=torch.int32, device=levels.device)
    c, b = ctypes.c_int32(), ctypes.c_int32()
    times = np.zeros(8, np.float32)
    check(lib().hesp_sim_autotune(platform.h, _ptr(cands), _ptr(levels), n_sample, max_tiles, max_level, task_cap,
                                  _ptr(ms), _ptr(st), _ptr(workspace), workspace.numel(),
                                  cache_path.encode() if cache_path else None, ctypes.byref(c), ctypes.byref(b),
                                  times.ctypes.data, _stream(stream)), "hesp_sim_autotune")
    return (c.value, b.value), times.tolist()


def sort_workspace(n_cand, device="cuda"):
    """Device workspace for sort_cands_by_size of up to n_cand candidates."""
    import torch
    sz = ctypes.c_size_t()
    check(lib().hesp_sort_cands_workspace_size(n_cand, ctypes.byref(sz)), "hesp_sort_cands_workspace_size")
    return torch.empty(sz.value, dtype=torch.uint8, device=device)


def sort_cands_by_size(cands, levels, n_cand, sorted_cands=None, perm=None, ws=None, stream=None):
    """Candidates reordered largest DAG first; returns (sorted_cands, perm)."""
    import torch
    sz = ctypes.c_size_t()
    check(lib().hesp_sort_cands_workspace_size(n_cand, ctypes.byref(sz)), "hesp_sort_cands_workspace_size")
    if ws is None:
        ws = torch.empty(sz.value, dtype=torch.uint8, device=levels.device)
    if sorted_cands is None:
        sorted_cands = torch.empty(n_cand * 16, dtype=torch.uint8, device=levels.device)
    if perm is None:
        perm = torch.empty(n_cand, dtype=torch.int32, device=levels.device)
    check(lib().hesp_sort_cands_by_size(_ptr(cands), _ptr(levels), n_cand, _ptr(sorted_cands), _ptr(perm), _ptr(ws),
                                        ws.numel(), _stream(stream)), "hesp_sort_cands_by_size")
    return sorted_cands, perm
