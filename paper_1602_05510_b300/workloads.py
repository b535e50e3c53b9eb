"""Seeded synthetic inputs: platform descriptions and candidate partition vectors.

This module holds the inputs only -- no part of the simulation's arithmetic
(no task times, no transfer times, no scheduling).  It is the one module shared
by the CUDA path's tests and the CPU oracle's tests.

Platforms follow the synthetic cost model of the workloads (HeSP, Sec. 2:
memory spaces, processors bound to memories, per-type performance models and a
transfer model; Sec. 3 models a CPU-GPU machine and a big.LITTLE board):

* a processor type has a peak rate (GFLOP/s), a half-performance size ``h`` and
  an efficiency per operation (chol, trsm, syrk, gemm) in percent;
* memory 0 is host memory; GPU-type processor g owns memory 1 + g;
* one transfer model for every pair of memories: latency + bytes / bandwidth.

Candidate partition vectors hold one split level per base task of the blocked
Cholesky loop (Fig. 1 order).  Random vectors come from SplitMix64 (Steele,
Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
used as a counter-based generator: output k of candidate c under a seed is
``mix(seed + ((c << 32) + k + 1) * 0x9E3779B97F4A7C15)``, and a draw in
[0, m) is Lemire's multiply-shift ``((u >> 32) * m) >> 32``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1

CHOL, TRSM, SYRK, GEMM = 0, 1, 2, 3

# Efficiencies in percent, ordered (chol, trsm, syrk, gemm): gemm 1.0,
# syrk 0.9, trsm 0.8, chol 0.35 on CPUs and 0.15 on GPUs.
CPU_EFF = (35, 80, 90, 100)
GPU_EFF = (15, 80, 90, 100)


@dataclass(frozen=True)
class ProcType:
    peak_gflops: int
    h: int
    eff_pct: Tuple[int, int, int, int]


@dataclass(frozen=True)
class PlatformSpec:
    name: str
    n_mem: int
    types: Tuple[ProcType, ...]
    procs: Tuple[Tuple[int, int], ...]  # (memory, type) per processor, in id order
    xfer_latency_ns: int = 8000
    bytes_per_elem: int = 8
    bw_bytes_per_ns: int = 12
    exec_overrides: Tuple[Tuple[int, int, int, int], ...] = field(default_factory=tuple)


CPU_TYPE = ProcType(30, 96, CPU_EFF)
GPU_TYPE = ProcType(2500, 768, GPU_EFF)
BIG_TYPE = ProcType(12, 64, CPU_EFF)
LITTLE_TYPE = ProcType(3, 32, CPU_EFF)


def cpu_gpu_platform(n_cpu: int, n_gpu: int, name: str = "") -> PlatformSpec:
    """n_cpu cores in host memory, then n_gpu GPU-type processors, each in its
    own memory (processor ids: CPUs first)."""
    procs = tuple([(0, 0)] * n_cpu + [(1 + g, 1) for g in range(n_gpu)])
    return PlatformSpec(name or "cpu%d_gpu%d" % (n_cpu, n_gpu), 1 + n_gpu,
                        (CPU_TYPE, GPU_TYPE), procs)


def big_little_platform() -> PlatformSpec:
    """4 big + 4 LITTLE cores sharing host memory (no transfers)."""
    procs = tuple([(0, 0)] * 4 + [(0, 1)] * 4)
    return PlatformSpec("big4_little4", 1, (BIG_TYPE, LITTLE_TYPE), procs)


def single_cpu_platform() -> PlatformSpec:
    return PlatformSpec("cpu1", 1, (CPU_TYPE,), ((0, 0),))


PLATFORMS = {
    "cfg0": cpu_gpu_platform(4, 1, "cpu4_gpu1"),
    "cfg1a": cpu_gpu_platform(12, 1, "cpu12_gpu1"),
    "cfg1b": big_little_platform(),
    "cfg2": cpu_gpu_platform(16, 2, "cpu16_gpu2"),
    "cfg3": cpu_gpu_platform(16, 2, "cpu16_gpu2"),
    "cfg4": cpu_gpu_platform(32, 2, "cpu32_gpu2"),
}


def base_count(n: int) -> int:
    """Base tasks of the n x n tiled Cholesky: n(n+1)(n+2)/6."""
    return n * (n + 1) * (n + 2) // 6


# ----------------------------------------------------------------------------
# SplitMix64 (published definition), vectorised over numpy uint64
# ----------------------------------------------------------------------------

def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """The first `count` outputs of the sequential SplitMix64 generator."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64_mix(np.uint64(seed & _M64) + k * np.uint64(GAMMA))


def counter_u64(seed: int, c: np.ndarray, k: np.ndarray) -> np.ndarray:
    c = np.asarray(c, dtype=np.uint64)
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = (c << np.uint64(32)) + k + np.uint64(1)
        return splitmix64_mix(np.uint64(seed & _M64) + ctr * np.uint64(GAMMA))


def draw(u: np.ndarray, m: int) -> np.ndarray:
    """Lemire multiply-shift: ((u >> 32) * m) >> 32, a value in [0, m)."""
    with np.errstate(over="ignore"):
        return ((u >> np.uint64(32)) * np.uint64(m)) >> np.uint64(32)


# ----------------------------------------------------------------------------
# Candidate partition vectors of the workloads
# ----------------------------------------------------------------------------

def exhaustive_levels(n_base: int = 10) -> np.ndarray:
    """All 2**n_base vectors: candidate c splits base task t once iff bit t of c."""
    c = np.arange(1 << n_base, dtype=np.int64)[:, None]
    t = np.arange(n_base, dtype=np.int64)[None, :]
    return ((c >> t) & 1).astype(np.int8)


def uniform_levels(seed: int, first: int, count: int, n_base: int, n_levels: int) -> np.ndarray:
    """level[c][t] = draw(n_levels) of output k = t of candidate first + c."""
    c = np.arange(first, first + count, dtype=np.uint64)[:, None]
    t = np.arange(n_base, dtype=np.uint64)[None, :]
    return draw(counter_u64(seed, c, t), n_levels).astype(np.int8)


def uniform_factors(seed: int, first: int, count: int, n_base: int, max_factor: int) -> np.ndarray:
    """Partition factors k (p = 1/k) per base task: 1 + draw(max_factor) of
    output k = t of candidate first + c."""
    return (uniform_levels(seed, first, count, n_base, max_factor) + 1).astype(np.int8)


# Non-dyadic workload: 8 x 8 tiles of b = 3072 = 12 * 256 (so that every mix
# of factors 1..4 tiles a block exactly), factors uniform in {1, 2, 3, 4}.
FACTOR_N, FACTOR_B, FACTOR_MAX = 8, 3072, 4

B_CHOICES = (512, 1024, 2048)


def uneven_candidates(seed: int, first: int, count: int):
    """Ragged batch: n = 4 + draw(29) (k = 0), b = {512, 1024, 2048}[draw(3)]
    (k = 1), level of base task t from r = draw(10) at k = 2 + t mapped
    0-4 -> 0, 5-7 -> 1, 8-9 -> 2.  Returns (n[C], b[C], offsets[C+1], levels)."""
    c = np.arange(first, first + count, dtype=np.uint64)
    n = (4 + draw(counter_u64(seed, c, np.uint64(0)), 29)).astype(np.int32)
    bi = draw(counter_u64(seed, c, np.uint64(1)), 3).astype(np.int64)
    b = np.asarray(B_CHOICES, np.int32)[bi]
    nb = n.astype(np.int64) * (n + 1) * (n + 2) // 6
    off = np.zeros(count + 1, np.int64)
    off[1:] = np.cumsum(nb)
    levels = np.zeros(int(off[-1]), np.int8)
    lut = np.array([0, 0, 0, 0, 0, 1, 1, 1, 2, 2], np.int8)
    for i in range(count):
        t = np.arange(nb[i], dtype=np.uint64)
        r = draw(counter_u64(seed, np.uint64(first + i), t + np.uint64(2)), 10)
        levels[off[i]:off[i + 1]] = lut[r.astype(np.int64)]
    return n, b, off, levels


@dataclass(frozen=True)
class Workload:
    name: str
    n_tiles: int
    b: int
    n_levels: int
    n_cand: int
    seed: int
    platforms: Tuple[str, ...]


WORKLOADS = {
    "cfg0": Workload("exhaustive_n3_b1024", 3, 1024, 2, 1024, 0, ("cfg0",)),
    "cfg1": Workload("random_n8_b2048_l3", 8, 2048, 3, 65536, 1, ("cfg1a", "cfg1b")),
    "cfg2": Workload("uneven_n4-32_b512-2048", 0, 0, 3, 16384, 2, ("cfg2",)),
    "cfg3": Workload("surrogate_n16_b2048_l3", 16, 2048, 3, 1 << 20, 3, ("cfg3",)),
    "cfg4": Workload("search_n32_b2048_l4", 32, 2048, 4, 4096, 4, ("cfg4",)),
}


def workload_levels(key: str, first: int = 0, count: int | None = None) -> np.ndarray:
    w = WORKLOADS[key]
    count = w.n_cand if count is None else count
    nb = base_count(w.n_tiles)
    if key == "cfg0":
        return exhaustive_levels(nb)[first:first + count]
    return uniform_levels(w.seed, first, count, nb, w.n_levels)


# ----------------------------------------------------------------------------
# Surrogate initial weights: He-uniform from SplitMix64 (parameter id c,
# element k in row-major order): w = (2 f - 1) * sqrt(6 / fan_in),
# f = (u >> 40) * 2^-24, all in float32.
# ----------------------------------------------------------------------------

def he_uniform(seed: int, pid: int, rows: int, cols: int, fan_in: int, cols_used: int | None = None) -> np.ndarray:
    cols_used = cols if cols_used is None else cols_used
    k = np.arange(rows * cols, dtype=np.uint64)
    u = counter_u64(seed, np.uint64(pid), k)
    f = ((u >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)
    bound = np.sqrt(np.float32(6.0) / np.float32(fan_in)).astype(np.float32)
    w = ((np.float32(2.0) * f - np.float32(1.0)) * bound).astype(np.float32).reshape(rows, cols)
    if cols_used < cols:
        w[:, cols_used:] = 0.0
    return w


def surrogate_init(seed: int, F: int, Fp: int, H: int):
    """Initial FP32 parameters (W1 [H, Fp], b1, W2 [H, H], b2, w3 [H], b3)."""
    return dict(W1=he_uniform(seed, 0, H, Fp, F, F), b1=np.zeros(H, np.float32),
                W2=he_uniform(seed, 1, H, H, H), b2=np.zeros(H, np.float32),
                w3=he_uniform(seed, 2, 1, H, H).reshape(H), b3=np.zeros(1, np.float32))


def mutants(parents: np.ndarray, n_levels: int, p_mut: float, seed: int, first: int, n: int) -> np.ndarray:
    """Proposal c copies parent c mod len(parents) and redraws each level with
    probability round(p_mut 2^16) / 2^16 (test at output k = 2t, new level at
    k = 2t + 1 of candidate first + c)."""
    parents = np.asarray(parents, np.int8)
    P, nb = parents.shape
    p_num = np.uint64(int(p_mut * 65536.0 + 0.5))
    c = np.arange(first, first + n, dtype=np.uint64)[:, None]
    t = np.arange(nb, dtype=np.uint64)[None, :]
    redraw = draw(counter_u64(seed, c, 2 * t), 65536) < p_num
    new = draw(counter_u64(seed, c, 2 * t + np.uint64(1)), n_levels).astype(np.int8)
    base = parents[np.arange(n) % P]
    return np.where(redraw, new, base).astype(np.int8)
