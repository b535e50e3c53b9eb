"""CPU oracle of the HeSP scheduling-partitioning simulation (arXiv 1602.05510).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its binding) never imports,
links or calls it, and it never imports them: the two share no code.  The only
module both sides use is the seeded input generator
``paper_1602_05510_b300.workloads``, which holds none of the method's
arithmetic.

The C file ``hesp_oracle.c`` is the oracle proper (plain, single-threaded, in
the order the paper describes the method: Fig. 1 base loop, Sec. 2.1
partitioners, dependences, performance / transfer models, FCFS + EFT-P with
write-back caching).  This module compiles it with gcc and wraps it with
ctypes and numpy.  ``mlp_ref`` holds the FP64 reference of the surrogate MLP;
``solver`` the iterative partition solver (Sec. 2.1 "Iterative solver") over
this simulation.

Every simulator function here is pinned by the tests in
``tests/test_oracle_*.py`` (closed forms, numerical execution of the DAG,
hand-derived worked examples, brute force, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hesp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OP_CHOL, OP_TRSM, OP_SYRK, OP_GEMM = 0, 1, 2, 3
OP_NAMES = ("chol", "trsm", "syrk", "gemm")
MAX_TYPES, MAX_PROCS, MAX_MEMS, MAX_OVR = 8, 64, 8, 256


def build(force: bool = False) -> str:
    """Compile hesp_oracle.c into liboracle.so (gcc -O2); returns the path."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
        return _LIB


class Platform(ctypes.Structure):
    _fields_ = [
        ("n_mem", ctypes.c_int32),
        ("n_types", ctypes.c_int32),
        ("peak_gflops", ctypes.c_int64 * MAX_TYPES),
        ("h", ctypes.c_int64 * MAX_TYPES),
        ("eff_pct", (ctypes.c_int32 * 4) * MAX_TYPES),
        ("n_procs", ctypes.c_int32),
        ("proc_mem", ctypes.c_int32 * MAX_PROCS),
        ("proc_type", ctypes.c_int32 * MAX_PROCS),
        ("xfer_latency_ns", ctypes.c_int64),
        ("bytes_per_elem", ctypes.c_int64),
        ("bw_bytes_per_ns", ctypes.c_int64),
        ("n_ovr", ctypes.c_int32),
        ("ovr_op", ctypes.c_int32 * MAX_OVR),
        ("ovr_type", ctypes.c_int32 * MAX_OVR),
        ("ovr_bs", ctypes.c_int64 * MAX_OVR),
        ("ovr_ns", ctypes.c_int64 * MAX_OVR),
        ("order", ctypes.c_int32),
        ("select", ctypes.c_int32),
        ("rp_seed", ctypes.c_uint64),
        ("cache", ctypes.c_int32),
        ("use_links", ctypes.c_int32),
        ("link_lat", (ctypes.c_int64 * MAX_MEMS) * MAX_MEMS),
        ("link_bw", (ctypes.c_int64 * MAX_MEMS) * MAX_MEMS),
        ("cap_bytes", ctypes.c_int64 * MAX_MEMS),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in
                ("makespan", "n_tasks", "n_events", "n_transfers", "xfer_elems", "atom_visits", "evicted",
                 "written_back")]


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


def build_variant(source_text: str, out_path: str) -> str:
    """Compile a variant of the oracle's C source (the tests plant a mistake
    in a copy of it and check that a pin fails) into out_path."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-w", "-shared", "-fPIC", "-o", out_path, src])
    return out_path


class using_library:
    """Context in which every oracle call of this module goes to the library
    at `path` (a variant built by build_variant) instead of liboracle.so."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = _load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _load(path):
    """The oracle library at `path` with its argument types declared."""
    L = ctypes.CDLL(path)
    i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    L.or_exec_ns.restype = i64
    L.or_exec_ns.argtypes = [ctypes.POINTER(Platform), i32, i32, i64]
    L.or_xfer_ns.restype = i64
    L.or_xfer_ns.argtypes = [ctypes.POINTER(Platform), i64]
    L.or_base_count.restype = i64
    L.or_base_count.argtypes = [i32]
    L.or_base_ops.restype = ctypes.c_int
    L.or_base_ops.argtypes = [i32, vp]
    L.or_levels_to_code.restype = i64
    L.or_levels_to_code.argtypes = [i32, vp, vp, i64]
    L.or_expand.restype = i64
    L.or_expand.argtypes = [i32, i64, vp, i64, i64, vp, vp, vp, vp, vp, vp]
    L.or_deps.restype = i64
    L.or_deps.argtypes = [i32, i64, vp, i64, i64, i32, i32, i64, vp, vp, vp]
    L.or_simulate.restype = i32
    L.or_simulate.argtypes = [ctypes.POINTER(Platform), i32, i64, vp, i64, i64, i32, i32,
                              vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
    L.or_simulate_levels.restype = i32
    L.or_simulate_levels.argtypes = [ctypes.POINTER(Platform), i32, i64, vp, i32, i32,
                                     vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
    L.or_deps_side.restype = i64
    L.or_deps_side.argtypes = [i32, i64, vp, i64, i64, i32, i64, i64, vp, vp, vp]
    L.or_factors_to_code.restype = i64
    L.or_factors_to_code.argtypes = [i32, vp, vp, i64]
    L.or_simulate_factors.restype = i32
    L.or_simulate_factors.argtypes = [ctypes.POINTER(Platform), i32, i64, vp, i32,
                                      vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
    L.or_simulate_many.restype = i32
    L.or_simulate_many.argtypes = [ctypes.POINTER(Platform), i32, i64, vp, i64, vp, vp, vp]
    return L


ORDER_FCFS, ORDER_PL = 0, 1
SELECT_EFT, SELECT_EIT, SELECT_FP, SELECT_RP = 0, 1, 2, 3
CACHE_WB, CACHE_WT, CACHE_WA = 0, 1, 2


def make_platform(desc, order: int = ORDER_FCFS, select: int = SELECT_EFT, rp_seed: int = 0,
                  cache: int = CACHE_WB, links=None, capacity=None) -> Platform:
    """Oracle platform from a plain description (a dict or an object with the
    fields of ``paper_1602_05510_b300.workloads.PlatformSpec``), with the
    task order (FCFS / PL), the processor selection (EFT-P / EIT-P / F-P /
    R-P), the seed of R-P's draws, the caching policy (WB / WT / WA),
    optionally per-link costs {(src, dst): (latency_ns, bytes_per_ns)} (the
    other pairs keep the platform's scalars) and finite capacities of
    accelerator memories {mem: bytes}."""
    g = (lambda k: desc[k]) if isinstance(desc, dict) else (lambda k: getattr(desc, k))
    pl = Platform()
    pl.n_mem = g("n_mem")
    types = g("types")
    pl.n_types = len(types)
    for i, t in enumerate(types):
        tg = (lambda k: t[k]) if isinstance(t, dict) else (lambda k: getattr(t, k))
        pl.peak_gflops[i] = tg("peak_gflops")
        pl.h[i] = tg("h")
        for o in range(4):
            pl.eff_pct[i][o] = tg("eff_pct")[o]
    procs = g("procs")
    pl.n_procs = len(procs)
    for i, (m, ty) in enumerate(procs):
        pl.proc_mem[i] = m
        pl.proc_type[i] = ty
    pl.xfer_latency_ns = g("xfer_latency_ns")
    pl.bytes_per_elem = g("bytes_per_elem")
    pl.bw_bytes_per_ns = g("bw_bytes_per_ns")
    ovr = g("exec_overrides") if (isinstance(desc, dict) and "exec_overrides" in desc) or \
        (not isinstance(desc, dict) and hasattr(desc, "exec_overrides")) else ()
    pl.n_ovr = len(ovr)
    for i, (op, ty, bs, ns) in enumerate(ovr):
        pl.ovr_op[i], pl.ovr_type[i], pl.ovr_bs[i], pl.ovr_ns[i] = op, ty, bs, ns
    pl.order, pl.select, pl.rp_seed, pl.cache = order, select, rp_seed, cache
    if links:
        pl.use_links = 1
        for s_ in range(MAX_MEMS):
            for d_ in range(MAX_MEMS):
                lat, bw = links.get((s_, d_), (pl.xfer_latency_ns, pl.bw_bytes_per_ns))
                pl.link_lat[s_][d_] = lat
                pl.link_bw[s_][d_] = bw
    for m, nbytes in (capacity or {}).items():
        pl.cap_bytes[m] = nbytes
    return pl


def exec_ns(pl: Platform, op: int, ptype: int, bs: int) -> int:
    return int(lib().or_exec_ns(ctypes.byref(pl), op, ptype, bs))


def xfer_ns(pl: Platform, elems: int) -> int:
    return int(lib().or_xfer_ns(ctypes.byref(pl), elems))


def base_count(n: int) -> int:
    return int(lib().or_base_count(n))


def base_ops(n: int) -> np.ndarray:
    out = np.zeros(base_count(n), np.int32)
    lib().or_base_ops(n, out.ctypes.data)
    return out


def levels_to_code(n: int, levels) -> np.ndarray:
    lv = np.ascontiguousarray(levels, np.int8)
    cap = int(sum(2 * 8 ** int(l) for l in lv)) + 1
    code = np.zeros(cap, np.int8)
    k = lib().or_levels_to_code(n, lv.ctypes.data, code.ctypes.data, cap)
    if k < 0:
        raise ValueError("bad levels (%d)" % k)
    return code[:k].copy()


def _cap_for_code(code) -> int:
    return max(1, int(len(code)))


def expand(n: int, b: int, code) -> dict:
    """Tasks of the DAG in creation order: op, depth, base, nreg, bs, regs[T,3,3]."""
    code = np.ascontiguousarray(code, np.int8)
    cap = _cap_for_code(code)
    op = np.zeros(cap, np.int32)
    depth = np.zeros(cap, np.int32)
    base = np.zeros(cap, np.int32)
    nreg = np.zeros(cap, np.int32)
    bs = np.zeros(cap, np.int64)
    regs = np.zeros(cap * 9, np.int64)
    T = lib().or_expand(n, b, code.ctypes.data, len(code), cap, op.ctypes.data, depth.ctypes.data,
                        base.ctypes.data, nreg.ctypes.data, bs.ctypes.data, regs.ctypes.data)
    if T < 0:
        raise ValueError("expand failed (%d)" % T)
    return dict(op=op[:T], depth=depth[:T], base=base[:T], nreg=nreg[:T], bs=bs[:T],
                regs=regs[:T * 9].reshape(T, 3, 3))


def deps(n: int, b: int, code, mode: int, atom_level: int = 0):
    """Predecessor lists: (pred_off[T+1], preds[E], war_edges).
    mode 0 = all pairs (definition), 1 = atoms of side b / 2**atom_level."""
    code = np.ascontiguousarray(code, np.int8)
    cap_t = _cap_for_code(code)
    T = len(expand(n, b, code)["op"])
    cap_e = 1 << 16
    while True:
        po = np.zeros(cap_t + 1, np.int64)
        pv = np.zeros(cap_e, np.int32)
        war = ctypes.c_int32(0)
        E = lib().or_deps(n, b, code.ctypes.data, len(code), cap_t, mode, atom_level, cap_e,
                          po.ctypes.data, pv.ctypes.data, ctypes.addressof(war))
        if E == -2 and cap_e < (1 << 30):
            cap_e *= 8
            continue
        if E < 0:
            raise ValueError("deps failed (%d)" % E)
        return po[:T + 1].copy(), pv[:E].copy(), int(war.value)


def factors_to_code(n: int, factors) -> np.ndarray:
    """Split code of one-level k-way partitions (Sec. 2.1, partition
    parameter p = 1 / factors[t] for base task t)."""
    fv = np.ascontiguousarray(factors, np.int8)
    cap = int(sum(1 + int(f) ** 3 for f in fv)) + 1
    code = np.zeros(cap, np.int8)
    k = lib().or_factors_to_code(n, fv.ctypes.data, code.ctypes.data, cap)
    if k < 0:
        raise ValueError("bad factors (%d)" % k)
    return code[:k].copy()


def lcm_of(factors) -> int:
    L = 1
    for f in np.asarray(factors, np.int64).reshape(-1):
        L = L * int(f) // int(np.gcd(L, int(f)))
    return L


def deps_side(n: int, b: int, code, atom_side: int):
    """Atom last-writer predecessor lists with atoms of side atom_side:
    (pred_off[T+1], preds[E], war_edges)."""
    code = np.ascontiguousarray(code, np.int8)
    cap_t = _cap_for_code(code)
    T = len(expand(n, b, code)["op"])
    cap_e = 1 << 16
    while True:
        po = np.zeros(cap_t + 1, np.int64)
        pv = np.zeros(cap_e, np.int32)
        war = ctypes.c_int32(0)
        E = lib().or_deps_side(n, b, code.ctypes.data, len(code), cap_t, 1, atom_side, cap_e,
                               po.ctypes.data, pv.ctypes.data, ctypes.addressof(war))
        if E == -2 and cap_e < (1 << 30):
            cap_e *= 8
            continue
        if E < 0:
            raise ValueError("deps failed (%d)" % E)
        return po[:T + 1].copy(), pv[:E].copy(), int(war.value)


def simulate_factors(pl: Platform, n: int, b: int, factors, dep_mode: int = 1, schedule: bool = True):
    """One candidate of one-level k-way partitions: factors[t] per base task
    (Fig. 1 order); atoms of side b / lcm(factors)."""
    fv = np.ascontiguousarray(factors, np.int8)
    cap = int(sum(int(f) ** 3 for f in fv)) + 1
    proc = np.zeros(cap, np.int16) if schedule else None
    start = np.zeros(cap, np.int64) if schedule else None
    fin = np.zeros(cap, np.int64) if schedule else None
    order = np.zeros(cap, np.int32) if schedule else None
    issue = np.zeros(cap, np.int64) if schedule else None
    st = Stats()
    rc = lib().or_simulate_factors(ctypes.byref(pl), n, b, fv.ctypes.data, dep_mode,
                                   proc.ctypes.data if schedule else None,
                                   start.ctypes.data if schedule else None,
                                   fin.ctypes.data if schedule else None,
                                   order.ctypes.data if schedule else None,
                                   issue.ctypes.data if schedule else None, ctypes.byref(st))
    return _result(rc, st, proc, start, fin, order, issue)


def simulate_code(pl: Platform, n: int, b: int, code, atom_level: int, dep_mode: int = 1,
                  schedule: bool = True):
    code = np.ascontiguousarray(code, np.int8)
    cap = _cap_for_code(code)
    proc = np.zeros(cap, np.int16) if schedule else None
    start = np.zeros(cap, np.int64) if schedule else None
    fin = np.zeros(cap, np.int64) if schedule else None
    order = np.zeros(cap, np.int32) if schedule else None
    issue = np.zeros(cap, np.int64) if schedule else None
    st = Stats()
    rc = lib().or_simulate(ctypes.byref(pl), n, b, code.ctypes.data, len(code), cap, atom_level, dep_mode,
                           proc.ctypes.data if schedule else None,
                           start.ctypes.data if schedule else None,
                           fin.ctypes.data if schedule else None,
                           order.ctypes.data if schedule else None,
                           issue.ctypes.data if schedule else None, ctypes.byref(st))
    return _result(rc, st, proc, start, fin, order, issue)


def _result(rc, st, proc, start, fin, order, issue):
    T = int(st.n_tasks)
    out = dict(status=int(rc), makespan=int(st.makespan), n_tasks=T, n_events=int(st.n_events),
               n_transfers=int(st.n_transfers), xfer_elems=int(st.xfer_elems),
               atom_visits=int(st.atom_visits), evicted=int(st.evicted), written_back=int(st.written_back))
    if proc is not None:
        out.update(proc=proc[:T].copy(), start=start[:T].copy(), finish=fin[:T].copy(),
                   order=order[:T].copy(), issue=issue[:T].copy())
    return out


def simulate(pl: Platform, n: int, b: int, levels, atom_level: int = -1, dep_mode: int = 1,
             schedule: bool = True):
    """One candidate: one split level per base task (Fig. 1 order)."""
    lv = np.ascontiguousarray(levels, np.int8)
    cap = int(sum(8 ** int(l) for l in lv)) + 1
    proc = np.zeros(cap, np.int16) if schedule else None
    start = np.zeros(cap, np.int64) if schedule else None
    fin = np.zeros(cap, np.int64) if schedule else None
    order = np.zeros(cap, np.int32) if schedule else None
    issue = np.zeros(cap, np.int64) if schedule else None
    st = Stats()
    rc = lib().or_simulate_levels(ctypes.byref(pl), n, b, lv.ctypes.data, atom_level, dep_mode,
                                  proc.ctypes.data if schedule else None,
                                  start.ctypes.data if schedule else None,
                                  fin.ctypes.data if schedule else None,
                                  order.ctypes.data if schedule else None,
                                  issue.ctypes.data if schedule else None, ctypes.byref(st))
    return _result(rc, st, proc, start, fin, order, issue)


def simulate_many(pl: Platform, n: int, b: int, levels: np.ndarray, threads: int = 1):
    """Many candidates of one (n, b); levels is [C, n_base] int8.  With
    threads > 1 the candidates are split into contiguous chunks run by Python
    threads (ctypes releases the GIL during each call)."""
    lv = np.ascontiguousarray(levels, np.int8)
    C = lv.shape[0]
    ms = np.zeros(C, np.int64)
    stt = np.zeros(C, np.int32)
    tasks = np.zeros(C, np.int64)
    L = lib()

    def run(a, b_):
        if b_ <= a:
            return
        L.or_simulate_many(ctypes.byref(pl), n, b, lv[a:b_].ctypes.data, b_ - a,
                           ms[a:].ctypes.data, stt[a:].ctypes.data, tasks[a:].ctypes.data)

    if threads <= 1:
        run(0, C)
    else:
        bounds = np.linspace(0, C, threads + 1).astype(int)
        ths = [threading.Thread(target=run, args=(int(bounds[i]), int(bounds[i + 1])))
               for i in range(threads)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    return ms, stt, tasks
