// Selection of the best-ranked proposals and the surrogate's error metrics.
//
// hesp_select_topk: the k smallest float keys of n (ties to the lowest index),
// returned in ascending index order, by a three-pass radix select on the
// order-preserving 32-bit image of the keys (11, 11, 10 bits), then an
// order-preserving compaction.
// hesp_make_cands: candidates pointing at selected rows of a level array.
// hesp_rank_metrics: mean relative makespan error of the surrogate and the
// Spearman rank correlation (average ranks for ties) between predicted and
// exact makespans.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hesp_internal.h"

namespace {

__device__ __forceinline__ uint32_t key_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

struct SelState {
    uint32_t prefix;    // digits found so far (high bits)
    uint32_t pmask;     // bits of the key fixed by the prefix
    int64_t remaining;  // rank still to find inside the current bucket (1-based)
    int64_t n_less;     // keys strictly below the threshold
};

// histogram of digit [shift, shift + bits) among keys matching the prefix
__global__ void hist_kernel(const float *keys, int64_t n, const SelState *st, int shift, int bits, uint32_t *hist) {
    __shared__ uint32_t sh[2048];
    const int nb = 1 << bits;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t prefix = st->prefix, pmask = st->pmask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t kb = key_bits(keys[i]);
        if ((kb & pmask) == prefix) atomicAdd(&sh[(kb >> shift) & (nb - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// pick the digit holding the remaining-th key; one thread
__global__ void pick_kernel(SelState *st, uint32_t *hist, int shift, int bits) {
    const int nb = 1 << bits;
    int64_t acc = 0;
    int d = 0;
    for (; d < nb; ++d) {
        if (acc + hist[d] >= st->remaining) break;
        acc += hist[d];
    }
    if (d >= nb) d = nb - 1;
    st->remaining -= acc;
    st->n_less += acc;
    st->prefix |= (uint32_t)d << shift;
    st->pmask |= (uint32_t)(nb - 1) << shift;
    for (int i = 0; i < nb; ++i) hist[i] = 0;
}

// per-block counts of keys below / equal to the threshold
__global__ void count_kernel(const float *keys, int64_t n, const SelState *st, int64_t chunk, int64_t *cnt_less,
                             int64_t *cnt_eq) {
    __shared__ int64_t sl[32], se[32];
    const uint32_t thr = st->prefix;
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    int64_t l = 0, e = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t kb = key_bits(keys[i]);
        l += kb < thr;
        e += kb == thr;
    }
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
        e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sl[threadIdx.x >> 5] = l;
        se[threadIdx.x >> 5] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t tl = 0, te = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tl += sl[w];
            te += se[w];
        }
        cnt_less[blockIdx.x] = tl;
        cnt_eq[blockIdx.x] = te;
    }
}

__global__ void scan_kernel(int64_t nblocks, int64_t *cnt_less, int64_t *cnt_eq) {
    int64_t a = 0, b = 0;
    for (int64_t i = 0; i < nblocks; ++i) {
        const int64_t x = cnt_less[i], y = cnt_eq[i];
        cnt_less[i] = a;
        cnt_eq[i] = b;
        a += x;
        b += y;
    }
}

// ordered compaction: key < thr, or key == thr among the first `need_eq` equal keys
__global__ void write_kernel(const float *keys, int64_t n, const SelState *st, int64_t chunk, int64_t k,
                             const int64_t *off_less, const int64_t *off_eq, int64_t *idx_out) {
    const uint32_t thr = st->prefix;
    const int64_t need_eq = k - st->n_less;
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    int64_t base_l = off_less[blockIdx.x], base_e = off_eq[blockIdx.x];
    const int lane = threadIdx.x & 31;
    // one warp walks the chunk in order (chunks are small)
    if (threadIdx.x >= 32) return;
    for (int64_t i0 = lo; i0 < hi; i0 += 32) {
        const int64_t i = i0 + lane;
        uint32_t kb = 0xFFFFFFFFu;
        bool valid = i < hi;
        if (valid) kb = key_bits(keys[i]);
        const bool less = valid && kb < thr, eq = valid && kb == thr;
        const unsigned ml = __ballot_sync(0xFFFFFFFFu, less), me = __ballot_sync(0xFFFFFFFFu, eq);
        const unsigned below = (1u << lane) - 1u;
        const int64_t rl = base_l + __popc(ml & below), re = base_e + __popc(me & below);
        // position in the output = keys before it that are selected
        const int64_t eq_taken_before = min(re, need_eq);
        if (less) idx_out[rl + eq_taken_before] = i;
        if (eq && re < need_eq) idx_out[rl + re] = i;
        base_l += __popc(ml);
        base_e += __popc(me);
    }
}

__global__ void cands_kernel(const int64_t *idx, int64_t k, int n_tiles, int b, int64_t n_base, hesp_cand *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    hesp_cand c;
    c.n_tiles = n_tiles;
    c.b = b;
    c.level_offset = idx[i] * n_base;
    out[i] = c;
}

__global__ void gather_rows_kernel(const int8_t *src, const int64_t *idx, int64_t k, int64_t width, int8_t *dst) {
    const int64_t r = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (r >= k) return;
    const int8_t *s = src + idx[r] * width;
    int8_t *d = dst + r * width;
    for (int64_t c = threadIdx.x; c < width; c += blockDim.x) d[c] = s[c];
}

__global__ void gather_float_kernel(const float *src, const int64_t *idx, int64_t k, float *dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) dst[i] = src[idx[i]];
}

// average rank (1-based) of x[i] among x[0..k): less + (equal + 1) / 2
__global__ void rank_kernel(const double *x, int64_t k, double *rank) {
    __shared__ double tile[1024];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double xi = i < k ? x[i] : 0.0;
    int64_t less = 0, eq = 0;
    for (int64_t j0 = 0; j0 < k; j0 += blockDim.x) {
        const int64_t j = j0 + threadIdx.x;
        tile[threadIdx.x] = j < k ? x[j] : 0.0;
        __syncthreads();
        const int64_t m = min((int64_t)blockDim.x, k - j0);
        for (int64_t q = 0; q < m; ++q) {
            const double v = tile[q];
            less += v < xi;
            eq += v == xi;
        }
        __syncthreads();
    }
    if (i < k) rank[i] = (double)less + (double)(eq + 1) / 2.0;
}

__global__ void prep_kernel(const float *pred, const int64_t *ms, int64_t k, double mu, double sigma, double *xp,
                            double *xt, double *rel) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const double pm = exp((double)pred[i] * sigma + mu);
    const double tm = (double)ms[i];
    xp[i] = (double)pred[i];
    xt[i] = tm;
    rel[i] = fabs(pm - tm) / tm;
}

// out = [mean rel, pearson(rp, rt)] (one block, deterministic)
__global__ void final_kernel(const double *rel, const double *rp, const double *rt, int64_t k, double *out) {
    __shared__ double s[3][1024];
    double a = 0, sp = 0, st = 0, spp = 0, stt = 0, spt = 0;
    for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
        a += rel[i];
        sp += rp[i];
        st += rt[i];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = sp;
    s[2][threadIdx.x] = st;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
        __syncthreads();
    }
    const double mp = s[1][0] / k, mt = s[2][0] / k, mrel = s[0][0] / k;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
        const double dp = rp[i] - mp, dt = rt[i] - mt;
        spp += dp * dp;
        stt += dt * dt;
        spt += dp * dt;
    }
    s[0][threadIdx.x] = spp;
    s[1][threadIdx.x] = stt;
    s[2][threadIdx.x] = spt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = mrel;
        out[1] = (s[0][0] > 0 && s[1][0] > 0) ? s[2][0] / sqrt(s[0][0] * s[1][0]) : 0.0;
    }
}

// out[0] = min makespan over candidates with status 0 (INT64_MAX if none),
// out[1] = their task count (one block, deterministic).
__global__ void best_kernel(const int64_t *ms, const int32_t *status, const int64_t *ntasks, int64_t n, int64_t *out) {
    __shared__ int64_t sm[1024], se[1024];
    int64_t m = INT64_MAX, e = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        if (status[i] == 0) {
            m = min(m, ms[i]);
            if (ntasks) e += ntasks[i];
        }
    sm[threadIdx.x] = m;
    se[threadIdx.x] = e;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sm[threadIdx.x] = min(sm[threadIdx.x], sm[threadIdx.x + o]);
            se[threadIdx.x] += se[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sm[0];
        out[1] = se[0];
    }
}

// out[0] = min makespan over candidates with status 0 (INT64_MAX if none),
// out[1] = first + the lowest index holding it (-1 if none); one block,
// two block reductions (the minimum, then the lowest index at it).
__global__ void best_index_kernel(const int64_t *ms, const int32_t *status, int64_t n, int64_t first, int64_t *out) {
    __shared__ int64_t sm[1024];
    __shared__ int64_t s_best;
    int64_t m = INT64_MAX;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        if (status[i] == 0) m = min(m, ms[i]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = min(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) s_best = sm[0];
    __syncthreads();
    const int64_t best = s_best;
    int64_t idx = INT64_MAX;
    if (best != INT64_MAX)
        for (int64_t i = threadIdx.x; i < n && idx == INT64_MAX; i += blockDim.x)
            if (status[i] == 0 && ms[i] == best) idx = i;
    __syncthreads();
    sm[threadIdx.x] = idx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = min(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = best;
        out[1] = best == INT64_MAX ? -1 : first + sm[0];
    }
}

constexpr int64_t kChunk = 4096;

}  // namespace

extern "C" {

int hesp_select_workspace_size(int64_t n, size_t *bytes) {
    if (n < 0 || !bytes) return HESP_ERR_ARG;
    const int64_t nblocks = (n + kChunk - 1) / kChunk;
    *bytes = 256 + 2048 * 4 + 2 * 8 * (size_t)(nblocks + 1);
    return HESP_OK;
}

int hesp_select_topk(const float *keys_dev, int64_t n, int64_t k, int64_t *idx_dev, void *ws, size_t ws_bytes,
                     void *stream) {
    if (!keys_dev || !idx_dev || !ws || n < 1 || k < 1 || k > n) return HESP_ERR_ARG;
    size_t need = 0;
    hesp_select_workspace_size(n, &need);
    if (ws_bytes < need || ((uintptr_t)ws & 15)) return HESP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    SelState *sst = (SelState *)w;
    uint32_t *hist = (uint32_t *)(w + 256);
    const int64_t nblocks = (n + kChunk - 1) / kChunk;
    int64_t *cl = (int64_t *)(w + 256 + 2048 * 4);
    int64_t *ce = cl + nblocks + 1;
    SelState init;
    init.prefix = 0;
    init.pmask = 0;
    init.remaining = k;
    init.n_less = 0;
    if (cudaMemcpyAsync(sst, &init, sizeof init, cudaMemcpyHostToDevice, st) != cudaSuccess) return HESP_ERR_CUDA;
    if (cudaMemsetAsync(hist, 0, 2048 * 4, st) != cudaSuccess) return HESP_ERR_CUDA;
    const int shifts[3] = {21, 10, 0}, bits[3] = {11, 11, 10};
    const unsigned g = (unsigned)min((int64_t)1184, (n + 255) / 256);
    for (int p = 0; p < 3; ++p) {
        hist_kernel<<<g, 256, 0, st>>>(keys_dev, n, sst, shifts[p], bits[p], hist);
        pick_kernel<<<1, 1, 0, st>>>(sst, hist, shifts[p], bits[p]);
    }
    count_kernel<<<(unsigned)nblocks, 256, 0, st>>>(keys_dev, n, sst, kChunk, cl, ce);
    scan_kernel<<<1, 1, 0, st>>>(nblocks, cl, ce);
    write_kernel<<<(unsigned)nblocks, 32, 0, st>>>(keys_dev, n, sst, kChunk, k, cl, ce, idx_dev);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int hesp_make_cands(const int64_t *idx_dev, int64_t k, int32_t n_tiles, int32_t b, hesp_cand *cands_dev,
                    void *stream) {
    if (!idx_dev || !cands_dev || k < 0 || n_tiles < 1) return HESP_ERR_ARG;
    if (k == 0) return HESP_OK;
    const int64_t nb = (int64_t)n_tiles * (n_tiles + 1) * (n_tiles + 2) / 6;
    cands_kernel<<<(unsigned)((k + 255) / 256), 256, 0, (cudaStream_t)stream>>>(idx_dev, k, n_tiles, b, nb,
                                                                                cands_dev);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int hesp_gather_f32(const float *src_dev, const int64_t *idx_dev, int64_t k, float *dst_dev, void *stream) {
    if (!src_dev || !idx_dev || !dst_dev || k < 0) return HESP_ERR_ARG;
    if (k == 0) return HESP_OK;
    gather_float_kernel<<<(unsigned)((k + 255) / 256), 256, 0, (cudaStream_t)stream>>>(src_dev, idx_dev, k, dst_dev);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int hesp_gather_rows(const int8_t *src_dev, const int64_t *idx_dev, int64_t k, int64_t width, int8_t *dst_dev,
                     void *stream) {
    if (!src_dev || !idx_dev || !dst_dev || k < 0 || width < 1) return HESP_ERR_ARG;
    if (k == 0) return HESP_OK;
    const int64_t gx = k < 65535 ? k : 65535;
    gather_rows_kernel<<<dim3((unsigned)gx, (unsigned)((k + gx - 1) / gx)), 128, 0, (cudaStream_t)stream>>>(
        src_dev, idx_dev, k, width, dst_dev);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int hesp_best_makespan(const int64_t *makespan_dev, const int32_t *status_dev, const int64_t *ntasks_dev, int64_t n,
                       int64_t *out_dev, void *stream) {
    if (!makespan_dev || !status_dev || !out_dev || n < 0) return HESP_ERR_ARG;
    best_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(makespan_dev, status_dev, ntasks_dev, n, out_dev);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int hesp_best_candidate(const int64_t *makespan_dev, const int32_t *status_dev, int64_t n, int64_t first_index,
                        int64_t *out_dev, void *stream) {
    if (!makespan_dev || !status_dev || !out_dev || n < 0 || first_index < 0) return HESP_ERR_ARG;
    best_index_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(makespan_dev, status_dev, n, first_index, out_dev);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int hesp_rank_metrics_workspace_size(int64_t k, size_t *bytes) {
    if (k < 0 || !bytes) return HESP_ERR_ARG;
    *bytes = (size_t)(5 * k + 2) * sizeof(double) + 256;
    return HESP_OK;
}

int hesp_rank_metrics(const float *pred_dev, const int64_t *makespan_dev, int64_t k, double mu, double sigma,
                      void *ws, size_t ws_bytes, double *out_host, void *stream) {
    if (!pred_dev || !makespan_dev || !ws || !out_host || k < 1 || !(sigma > 0)) return HESP_ERR_ARG;
    size_t need = 0;
    hesp_rank_metrics_workspace_size(k, &need);
    if (ws_bytes < need || ((uintptr_t)ws & 7)) return HESP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *xp = (double *)ws, *xt = xp + k, *rel = xt + k, *rp = rel + k, *rt = rp + k, *out = rt + k;
    const unsigned gb = (unsigned)((k + 255) / 256);
    prep_kernel<<<gb, 256, 0, st>>>(pred_dev, makespan_dev, k, mu, sigma, xp, xt, rel);
    rank_kernel<<<(unsigned)((k + 1023) / 1024), 1024, 0, st>>>(xp, k, rp);
    rank_kernel<<<(unsigned)((k + 1023) / 1024), 1024, 0, st>>>(xt, k, rt);
    final_kernel<<<1, 1024, 0, st>>>(rel, rp, rt, k, out);
    if (cudaMemcpyAsync(out_host, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return HESP_ERR_CUDA;
    return HESP_OK;
}

}  // extern "C"
