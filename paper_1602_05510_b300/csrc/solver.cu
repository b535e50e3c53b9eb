// HeSP's iterative partition solver (Sec. 2.1 "Iterative solver") on the
// device: the partition stage's candidate moves, and the score / sampling /
// apply step.  The schedule stage is the batched simulator: the current
// partition (hesp_simulate_critical, for the CP flags and its makespan) and
// every moved partition (hesp_simulate_batch, one launch for the whole
// neighbourhood), so each move is scored by its exact makespan gain.
//
// A partition is one value per base task in [lo, hi]: its split level
// (dyadic partitions, lo = 0) or its partition factor k (p = 1/k, lo = 1);
// move k = 2 t + d changes base task t by +1 (d = 0, partition finer) or -1
// (d = 1, merge back / repartition coarser).  Candidate moves, in increasing
// k: a finer move for each base task picked by the selection policy (All:
// every one; CP: those flagged critical; Shallow: those at the minimal
// value) that is below hi, and a coarser move for every base task above lo.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hesp_internal.h"

namespace hesp {
namespace {

constexpr int kThreads = 1024;
constexpr unsigned FULL = 0xFFFFFFFFu;

// Block-wide exclusive scan of one int per thread; returns the block total.
__device__ int block_excl_scan(int v, int *excl, int *s_warp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        s_warp[lane] = s;  // inclusive per warp
    }
    __syncthreads();
    const int before = w > 0 ? s_warp[w - 1] : 0;
    const int total = s_warp[31];
    *excl = before + x - v;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kThreads) moves_kernel(const int8_t *lv, int nb, int lo, int hi, int mode,
                                                         const int8_t *crit, int32_t *moves, int64_t *count) {
    __shared__ int s_warp[32];
    __shared__ int s_min;
    if (threadIdx.x == 0) s_min = 127;
    __syncthreads();
    if (mode == HESP_SOLVER_SHALLOW) {
        int m = 127;
        for (int t = threadIdx.x; t < nb; t += kThreads) m = min(m, (int)lv[t]);
        m = __reduce_min_sync(FULL, m);
        if ((threadIdx.x & 31) == 0) atomicMin(&s_min, m);
        __syncthreads();
    }
    const int lmin = s_min;
    int run = 0;
    for (int k0 = 0; k0 < 2 * nb; k0 += kThreads) {
        const int k = k0 + threadIdx.x;
        int ok = 0;
        if (k < 2 * nb) {
            const int t = k >> 1;
            const int l = lv[t];
            if (k & 1) {
                ok = l > lo;
            } else {
                const bool sel = mode == HESP_SOLVER_ALL || (mode == HESP_SOLVER_CP && crit[t] != 0) ||
                                 (mode == HESP_SOLVER_SHALLOW && l == lmin);
                ok = sel && l < hi;
            }
        }
        int excl;
        const int total = block_excl_scan(ok, &excl, s_warp);
        if (ok) moves[run + excl] = k;
        run += total;
    }
    if (threadIdx.x == 0) *count = run;
}

// Row r of the neighbourhood: the current partition with move moves[r] applied.
__global__ void rows_kernel(const int8_t *lv, int nb, const int32_t *moves, const int64_t *count, int8_t *rows) {
    const int64_t r = blockIdx.y;
    if (r >= *count) return;
    const int k = moves[r];
    const int t = k >> 1;
    const int d = (k & 1) ? -1 : 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x)
        rows[r * nb + i] = (int8_t)(lv[i] + (i == t ? d : 0));
}

// Score = current makespan - moved makespan, kept when positive (and the
// simulation succeeded).  Hard: the largest score, ties to the lower index.
// Soft: r = floor(u * S / 2^64), S = the kept scores' sum, u = SplitMix64
// (seed, c = iteration, k = 0); the first kept move whose running sum
// exceeds r.  The chosen move is applied to the partition in place.
__global__ void __launch_bounds__(kThreads) pick_kernel(const int64_t *ms, const int32_t *st, const int32_t *moves,
                                                        const int64_t *count, int pick, uint64_t seed,
                                                        int64_t iteration, int64_t *cur_ms, int8_t *lv,
                                                        int64_t *chosen) {
    __shared__ unsigned long long s_hi, s_lo, s_best;
    __shared__ int s_idx;
    __shared__ uint64_t s_part[32];
    const int64_t n = *count;
    const int64_t m = *cur_ms;
    if (threadIdx.x == 0) {
        s_hi = 0;
        s_lo = 0;
        s_best = 0;
        s_idx = INT32_MAX;
    }
    __syncthreads();
    auto score = [&](int64_t i) -> uint64_t {
        const int64_t g = m - ms[i];
        return (st[i] == HESP_OK && g > 0) ? (uint64_t)g : 0ull;
    };
    if (pick == HESP_PICK_HARD) {
        uint64_t best = 0;
        for (int64_t i = threadIdx.x; i < n; i += kThreads) best = max(best, score(i));
        const unsigned hi = __reduce_max_sync(FULL, (unsigned)(best >> 32));
        const unsigned lo = __reduce_max_sync(FULL, (unsigned)(best >> 32) == hi ? (unsigned)best : 0u);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_best, ((unsigned long long)hi << 32) | lo);
        __syncthreads();
        const uint64_t b = s_best;
        int idx = INT32_MAX;
        if (b > 0)
            for (int64_t i = threadIdx.x; i < n; i += kThreads)
                if (score(i) == b) {
                    idx = (int)i;
                    break;
                }
        idx = __reduce_min_sync(FULL, idx);
        if ((threadIdx.x & 31) == 0) atomicMin(&s_idx, idx);
        __syncthreads();
    } else {
        // S as a 128-bit sum (each score < 2^57; at most 2^31 moves)
        uint64_t lo = 0, hi = 0;
        for (int64_t i = threadIdx.x; i < n; i += kThreads) {
            const uint64_t v = score(i);
            lo += v;
            hi += lo < v;
        }
        atomicAdd(&s_hi, (unsigned long long)hi);
        const unsigned long long old = atomicAdd(&s_lo, (unsigned long long)lo);
        if (old + lo < old) atomicAdd(&s_hi, 1ull);
        __syncthreads();
        if (s_hi != 0) {  // S >= 2^64: not representable in the draw
            if (threadIdx.x == 0) *chosen = -2;
            return;
        }
        const uint64_t S = s_lo;
        if (S > 0) {
            const uint64_t r = __umul64hi(sm64_at(seed, (uint64_t)iteration, 0), S);
            // running sums in index order, one chunk of kThreads at a time
            uint64_t run = 0;
            for (int64_t i0 = 0; i0 < n; i0 += kThreads) {
                const int64_t i = i0 + threadIdx.x;
                const uint64_t v = i < n ? score(i) : 0;
                uint64_t x = v;
                const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint64_t y = __shfl_up_sync(FULL, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) s_part[w] = x;
                __syncthreads();
                if (w == 0) {
                    uint64_t s = s_part[lane];
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint64_t y = __shfl_up_sync(FULL, s, o);
                        if (lane >= o) s += y;
                    }
                    s_part[lane] = s;
                }
                __syncthreads();
                const uint64_t incl = run + (w > 0 ? s_part[w - 1] : 0) + x;
                int idx = (v > 0 && incl > r) ? (int)i : INT32_MAX;
                idx = __reduce_min_sync(FULL, idx);
                if (lane == 0) atomicMin(&s_idx, idx);
                const uint64_t total = s_part[31];
                __syncthreads();
                if (s_idx != INT32_MAX) break;
                run += total;
            }
        }
    }
    if (threadIdx.x == 0) {
        const int idx = s_idx;
        if (idx == INT32_MAX) {
            *chosen = -1;
        } else {
            const int k = moves[idx];
            lv[k >> 1] += (k & 1) ? -1 : 1;
            *cur_ms = ms[idx];
            *chosen = k;
        }
    }
}

}  // namespace
}  // namespace hesp

extern "C" int hesp_solver_moves_range(const int8_t *values_dev, int32_t n_base, int32_t lo, int32_t hi,
                                       int32_t mode, const int8_t *crit_dev, int32_t *moves_dev, int64_t *count_dev,
                                       int8_t *rows_dev, void *stream) {
    const int8_t *levels_dev = values_dev;
    if (!levels_dev || !moves_dev || !count_dev || n_base < 1 || lo < 0 || hi < lo || hi > 127 ||
        mode < HESP_SOLVER_ALL || mode > HESP_SOLVER_SHALLOW || (mode == HESP_SOLVER_CP && !crit_dev))
        return HESP_ERR_ARG;
    if (n_base > 32767) return HESP_ERR_UNSUPPORTED;  // one grid row per move
    const cudaStream_t st = (cudaStream_t)stream;
    hesp::moves_kernel<<<1, hesp::kThreads, 0, st>>>(levels_dev, n_base, lo, hi, mode, crit_dev, moves_dev,
                                                     count_dev);
    if (rows_dev) {
        const int bx = (n_base + 255) / 256;
        hesp::rows_kernel<<<dim3(bx, 2 * n_base), 256, 0, st>>>(levels_dev, n_base, moves_dev, count_dev, rows_dev);
    }
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

extern "C" int hesp_solver_moves(const int8_t *levels_dev, int32_t n_base, int32_t n_levels, int32_t mode,
                                 const int8_t *crit_dev, int32_t *moves_dev, int64_t *count_dev, int8_t *rows_dev,
                                 void *stream) {
    if (n_levels < 1 || n_levels > HESP_MAX_LEVEL + 1) return HESP_ERR_ARG;
    return hesp_solver_moves_range(levels_dev, n_base, 0, n_levels - 1, mode, crit_dev, moves_dev, count_dev,
                                   rows_dev, stream);
}

extern "C" int hesp_solver_pick(const int64_t *makespan_dev, const int32_t *status_dev, const int32_t *moves_dev,
                                const int64_t *count_dev, int32_t pick, uint64_t seed, int64_t iteration,
                                int64_t *cur_makespan_dev, int8_t *levels_dev, int64_t *chosen_dev, void *stream) {
    if (!makespan_dev || !status_dev || !moves_dev || !count_dev || !cur_makespan_dev || !levels_dev ||
        !chosen_dev || (pick != HESP_PICK_HARD && pick != HESP_PICK_SOFT) || iteration < 0)
        return HESP_ERR_ARG;
    hesp::pick_kernel<<<1, hesp::kThreads, 0, (cudaStream_t)stream>>>(makespan_dev, status_dev, moves_dev, count_dev,
                                                                      pick, seed, iteration, cur_makespan_dev,
                                                                      levels_dev, chosen_dev);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}
