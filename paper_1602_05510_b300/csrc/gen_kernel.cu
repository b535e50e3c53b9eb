// On-device candidate generation: partition vectors from SplitMix64 used as a
// counter-based generator (Steele, Lea, Flood, OOPSLA 2014): output k of
// candidate c is mix(seed + ((c << 32) + k + 1) * 0x9E3779B97F4A7C15), and a
// draw in [0, m) is Lemire's multiply-shift ((u >> 32) * m) >> 32.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hesp_internal.h"

namespace hesp {
namespace {

__device__ __forceinline__ uint32_t draw(uint64_t u, uint32_t m) { return lemire_draw(u, m); }

// One block row of threads per candidate tile of the level array.
__global__ void gen_fixed_kernel(int kind, uint64_t seed, int64_t first, int64_t n_cand, int nb, int n_levels,
                                 int n_tiles, int b, hesp_cand *cands, int8_t *levels) {
    const int64_t c = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (c >= n_cand) return;
    const uint64_t cg = (uint64_t)(first + c);
    int8_t *row = levels + c * nb;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        int lv;
        if (kind == HESP_GEN_EXHAUSTIVE) lv = t < 63 ? (int)((cg >> t) & 1u) : 0;
        else lv = (int)draw(sm64_at(seed, cg, (uint64_t)t), (uint32_t)n_levels);
        row[t] = (int8_t)lv;
    }
    if (threadIdx.x == 0 && cands) {
        hesp_cand cd;
        cd.n_tiles = n_tiles;
        cd.b = b;
        cd.level_offset = c * nb;
        cands[c] = cd;
    }
}

__global__ void uneven_shape_kernel(uint64_t seed, int64_t first, int64_t n_cand, hesp_cand *cands) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cand) return;
    const uint64_t cg = (uint64_t)(first + c);
    const int n = 4 + (int)draw(sm64_at(seed, cg, 0), 29);
    const int bsel = (int)draw(sm64_at(seed, cg, 1), 3);
    hesp_cand cd;
    cd.n_tiles = n;
    cd.b = 512 << bsel;
    cd.level_offset = (int64_t)n * (n + 1) * (n + 2) / 6;  // count; prefix-summed next
    cands[c] = cd;
}

// Exclusive prefix sum of the per-candidate base counts (one block).
__global__ void uneven_scan_kernel(int64_t n_cand, hesp_cand *cands, int64_t levels_cap, int64_t *levels_used) {
    __shared__ int64_t part[1024];
    const int tid = threadIdx.x;
    const int64_t chunk = (n_cand + blockDim.x - 1) / blockDim.x;
    const int64_t lo = tid * chunk, hi = min(n_cand, lo + chunk);
    int64_t s = 0;
    for (int64_t c = lo; c < hi; ++c) s += cands[c].level_offset;
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
        *levels_used = run <= levels_cap ? run : -1;
    }
    __syncthreads();
    int64_t run = part[tid];
    for (int64_t c = lo; c < hi; ++c) {
        const int64_t v = cands[c].level_offset;
        cands[c].level_offset = run;
        run += v;
    }
}

__global__ void uneven_fill_kernel(uint64_t seed, int64_t first, int64_t n_cand, const hesp_cand *cands,
                                   int8_t *levels, const int64_t *levels_used) {
    if (*levels_used < 0) return;
    const int64_t c = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (c >= n_cand) return;
    const uint64_t cg = (uint64_t)(first + c);
    const hesp_cand cd = cands[c];
    const int nb = cd.n_tiles * (cd.n_tiles + 1) * (cd.n_tiles + 2) / 6;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const uint32_t r = draw(sm64_at(seed, cg, (uint64_t)t + 2), 10);
        levels[cd.level_offset + t] = (int8_t)(r < 5 ? 0 : (r < 8 ? 1 : 2));
    }
}

// Mutants of parent partition vectors: proposal c copies parent
// (c mod n_parents) and redraws each level with probability p_num / 2^16
// (draw at k = 2 t from SplitMix64(seed, first + c); new level at k = 2 t + 1).
__global__ void mutate_kernel(const int8_t *parents, int n_parents, int nb, int n_levels, uint32_t p_num,
                              uint64_t seed, int64_t first, int64_t n, int8_t *out) {
    const int64_t c = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (c >= n) return;
    const uint64_t cg = (uint64_t)(first + c);
    const int8_t *par = parents + (c % n_parents) * (int64_t)nb;
    int8_t *row = out + c * nb;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        int8_t v = par[t];
        if (draw(sm64_at(seed, cg, 2 * (uint64_t)t), 65536u) < p_num)
            v = (int8_t)draw(sm64_at(seed, cg, 2 * (uint64_t)t + 1), (uint32_t)n_levels);
        row[t] = v;
    }
}

// Task count of each candidate (one warp per candidate) -> descending-size
// bucket key (65535 - min(65535, T / 16)).
__constant__ int32_t c_cnt_g[4][HESP_MAX_LEVEL + 1] = {
    {1, 4, 20, 120, 816}, {1, 6, 40, 288, 2176}, {1, 6, 40, 288, 2176}, {1, 8, 64, 512, 4096}};

__device__ int base_op(int n, int64_t t) {
    for (int k = 0; k < n; ++k) {
        const int64_t m = n - k - 1;
        const int64_t S = 1 + 2 * m + (m * (m - 1)) / 2;
        if (t < S) {
            if (t == 0) return 0;
            if (t <= m) return 1;
            t -= m + 1;
            for (int i = k + 1; i < n; ++i) {
                const int blk = n - i;
                if (t < blk) return t < blk - 1 ? 3 : 2;
                t -= blk;
            }
            return 2;
        }
        t -= S;
    }
    return 0;
}

__global__ void size_key_kernel(const hesp_cand *cands, const int8_t *levels, int64_t n_cand, uint32_t *key,
                                uint32_t *hist) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n_cand) return;
    const hesp_cand cd = cands[c];
    const int n = cd.n_tiles;
    int64_t T = 0;
    if (n >= 1 && n <= HESP_MAX_TILES) {
        const int64_t nb = (int64_t)n * (n + 1) * (n + 2) / 6;
        for (int64_t t = lane; t < nb; t += 32) {
            const int l = levels[cd.level_offset + t];
            T += (l >= 0 && l <= HESP_MAX_LEVEL) ? c_cnt_g[base_op(n, t)][l] : 1;
        }
    }
    for (int o = 16; o > 0; o >>= 1) T += __shfl_xor_sync(0xFFFFFFFFu, T, o);
    if (lane == 0) {
        const uint32_t k = 65535u - (uint32_t)min((int64_t)65535, T >> 4);
        key[c] = k;
        atomicAdd(&hist[k], 1u);
    }
}

__global__ void bucket_scan_kernel(uint32_t *hist) {
    // exclusive scan of 65,536 counters by one block of 1,024 threads
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x;
    uint32_t s = 0;
    for (int i = 0; i < 64; ++i) s += hist[t * 64 + i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        uint32_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const uint32_t v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    uint32_t run = part[t];
    for (int i = 0; i < 64; ++i) {
        const uint32_t v = hist[t * 64 + i];
        hist[t * 64 + i] = run;
        run += v;
    }
}

__global__ void bucket_scatter_kernel(const hesp_cand *in, int64_t n_cand, const uint32_t *key, uint32_t *cursor,
                                      hesp_cand *out, int32_t *perm) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cand) return;
    const uint32_t pos = atomicAdd(&cursor[key[c]], 1u);
    out[pos] = in[c];
    if (perm) perm[pos] = (int32_t)c;
}

dim3 cand_grid(int64_t n_cand) {
    const int64_t gx = n_cand < 65535 ? n_cand : 65535;
    return dim3((unsigned)gx, (unsigned)((n_cand + gx - 1) / gx));
}

}  // namespace

int launch_generate(int32_t kind, uint64_t seed, int64_t first, int64_t n_cand, int32_t n_tiles, int32_t b,
                    int32_t n_levels, hesp_cand *cands, int8_t *levels, cudaStream_t stream) {
    if (n_cand == 0) return HESP_OK;
    const int nb = n_tiles * (n_tiles + 1) * (n_tiles + 2) / 6;
    gen_fixed_kernel<<<cand_grid(n_cand), 128, 0, stream>>>(kind, seed, first, n_cand, nb, n_levels, n_tiles, b,
                                                             cands, levels);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int launch_mutate(const int8_t *parents, int32_t n_parents, int32_t n_base, int32_t n_levels, uint32_t p_num,
                  uint64_t seed, int64_t first, int64_t n, int8_t *out, cudaStream_t stream) {
    if (n == 0) return HESP_OK;
    mutate_kernel<<<cand_grid(n), 128, 0, stream>>>(parents, n_parents, n_base, n_levels, p_num, seed, first, n, out);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int launch_sort_by_size(const hesp_cand *in, const int8_t *levels, int64_t n, hesp_cand *out, int32_t *perm,
                        void *ws, cudaStream_t st) {
    if (n == 0) return HESP_OK;
    uint32_t *hist = (uint32_t *)ws;
    uint32_t *key = hist + 65536;
    if (cudaMemsetAsync(hist, 0, 65536 * 4, st) != cudaSuccess) return HESP_ERR_CUDA;
    size_key_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(in, levels, n, key, hist);
    bucket_scan_kernel<<<1, 1024, 0, st>>>(hist);
    bucket_scatter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, n, key, hist, out, perm);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int launch_generate_uneven(uint64_t seed, int64_t first, int64_t n_cand, hesp_cand *cands, int8_t *levels,
                           int64_t levels_cap, int64_t *levels_used, cudaStream_t stream) {
    if (n_cand == 0) return cudaMemsetAsync(levels_used, 0, sizeof(int64_t), stream) == cudaSuccess
                                ? HESP_OK
                                : HESP_ERR_CUDA;
    uneven_shape_kernel<<<(unsigned)((n_cand + 255) / 256), 256, 0, stream>>>(seed, first, n_cand, cands);
    uneven_scan_kernel<<<1, 1024, 0, stream>>>(n_cand, cands, levels_cap, levels_used);
    uneven_fill_kernel<<<cand_grid(n_cand), 128, 0, stream>>>(seed, first, n_cand, cands, levels, levels_used);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

}  // namespace hesp
