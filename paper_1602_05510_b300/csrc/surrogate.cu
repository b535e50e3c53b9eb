// Learned surrogate of the simulator: an MLP  F -> H -> H -> 1  (ReLU, bf16
// weights and activations, FP32 accumulation on the tensor cores) mapping a
// one-hot encoded partition vector to a standardised log-makespan.  Trained on
// the GPU with the project's own forward / backward kernels and Adam; ranks
// large proposal sets, whose best slice is re-simulated exactly.
//
// Layer math (one batch of B rows):
//   X   = one_hot(levels)                   [B, Fp]  (F = n_base * n_levels, Fp = F rounded up to 64;
//                                                  built tile by tile inside the layer-1 GEMM)
//   A1  = bf16(relu(X W1^T + b1))           [B, H]   GEMM epilogue 1 (+ A1^T)
//   A2  = bf16(relu(A1 W2^T + b2))          [B, H]   GEMM epilogue 1
//   y   = A2 w3 + b3,  t = (ln makespan - mu) / sigma,  L = mean (y - t)^2
//   dy  = 2 (y - t) / B;  dw3 = A2^T dy;  db3 = sum dy
//   dZ2 = bf16(dy w3^T * [A2 > 0])  (+ dZ2^T);  dW2 = dZ2^T A1;  db2 = sum_b dZ2
//   dZ1 = bf16((dZ2 W2) * [A1 > 0]) (+ dZ1^T);  dW1 = dZ1^T X;   db1 = sum_b dZ1
//   Adam on FP32 masters, then bf16 copies W1, W2 and W2^T for the next GEMMs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hesp_internal.h"


using namespace hesp;

struct hesp_surrogate {
    int32_t n_base, n_levels, H, max_batch;
    int64_t F, Fp;
    uint64_t seed;
    int64_t step;      // Adam steps taken
    double mu, sigma;  // target standardisation
    // FP32 masters, gradients, Adam moments: one block per tensor
    float *W1, *b1, *W2, *b2, *w3, *b3;
    float *gW1, *gb1, *gW2, *gb2, *gw3, *gb3;
    float *mW1, *mb1, *mW2, *mb2, *mw3, *mb3;
    float *vW1, *vb1, *vW2, *vb2, *vw3, *vb3;
    __nv_bfloat16 *W1b, *W2b, *W2Tb;  // bf16 copies for the GEMMs
    // activations for up to max_batch rows
    int8_t *lv;        // gathered levels [B, n_base]
    int64_t *ms;       // gathered makespans [B]
    __nv_bfloat16 *XT, *A1, *A1T, *A2, *dZ2, *dZ2T, *dZ1, *dZ1T;
    int8_t *lvp;  // levels with rows padded to ldp bytes, for the layer-1 GEMM
    int64_t ldp;
    float *y, *dy, *sq, *loss;
    int32_t *err;
    void *mem;  // one device allocation holding all of the above
};

namespace {


// He-uniform initialisation: w = (2 f - 1) * bound, f = (u >> 40) 2^-24.
__global__ void init_uniform_kernel(float *w, int64_t rows, int64_t cols, int64_t cols_used, uint64_t seed,
                                    uint64_t pid, float bound) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i % cols;
        const uint64_t u = sm64_at(seed, pid, (uint64_t)i);
        const float f = (float)(u >> 40) * 5.9604644775390625e-8f;  // 2^-24
        w[i] = c < cols_used ? __fmul_rn(__fsub_rn(__fmul_rn(2.0f, f), 1.0f), bound) : 0.0f;
    }
}

__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, __nv_bfloat16 *dst_t, int64_t rows,
                               int64_t cols) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols;
         i += (int64_t)gridDim.x * blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(src[i]);
        dst[i] = h;
        if (dst_t) dst_t[(i % cols) * rows + i / cols] = h;
    }
}

// Copy B rows of n_base level bytes (row stride `stride`) into rows of ldp
// bytes (a multiple of 16), the layout the layer-1 GEMM reads with TMA.
__global__ void pad_levels_kernel(const int8_t *lv, int64_t stride, int B, int n_base, int ldp, int8_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B * n_base;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / n_base, t = i - b * n_base;
        out[b * ldp + t] = lv[b * stride + t];
    }
}

// XT[f, b] = X[b, f] = (levels[b, f / NL] == f % NL), the transposed one-hot
// matrix of the weight-gradient GEMM: one thread writes 8 rows-of-b (16 bytes)
// of one feature.  (The forward pass never materialises X: layer 1 builds
// its A tiles from the levels inside the GEMM.)
__global__ void onehot_t_kernel(const int8_t *lv, int lv_stride, int B, int n_base, int NL, int Fp,
                                __nv_bfloat16 *XT) {
    const int chunks = B >> 3;
    const int64_t total = (int64_t)Fp * chunks;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(i / chunks), b0 = (int)(i % chunks) << 3;
        const int t = f / NL, v = f - t * NL;
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            const bool a = t < n_base && lv[(int64_t)(b0 + q) * lv_stride + t] == v;
            const bool c = t < n_base && lv[(int64_t)(b0 + q + 1) * lv_stride + t] == v;
            w[q >> 1] = (a ? 0x3F80u : 0u) | ((c ? 0x3F80u : 0u) << 16);
        }
        *reinterpret_cast<uint4 *>(XT + (int64_t)f * B + b0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// One warp per row: y = A2[b] . w3 + b3; with targets, dy and the row's
// squared error (summed by loss_kernel in a fixed order).
__global__ void l3_kernel(const __nv_bfloat16 *A2, int H, const float *w3, const float *b3, int B, float *y,
                          const int64_t *ms, double mu, double sigma, float *dy, float *sq) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= B) return;
    float s = 0.f;
    for (int k = lane; k < H; k += 32) s = fmaf(__bfloat162float(A2[(int64_t)warp * H + k]), w3[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    const float yy = s + b3[0];
    if (lane == 0) {
        y[warp] = yy;
        if (ms) {
            const float t = (float)((log((double)ms[warp]) - mu) / sigma);
            const float d = yy - t;
            dy[warp] = 2.f * d / (float)B;
            sq[warp] = d * d;
        }
    }
}

// loss = mean of sq[0 .. B), one block in a fixed order (deterministic).
__global__ void loss_kernel(const float *sq, int B, float *loss) {
    __shared__ float part[1024];
    float s = 0.f;
    for (int i = threadIdx.x; i < B; i += blockDim.x) s += sq[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)B;
}

// dZ2 = bf16(dy w3^T * [A2 > 0]) and its transpose, 32 x 32 tiles.
__global__ void dz2_kernel(const __nv_bfloat16 *A2, const float *dy, const float *w3, int B, int H,
                           __nv_bfloat16 *dZ2, __nv_bfloat16 *dZ2T) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int b0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int b = b0 + r, k = k0 + threadIdx.x;
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (b < B && k < H) {
            const float a = __bfloat162float(A2[(int64_t)b * H + k]);
            v = __float2bfloat16_rn(a > 0.f ? dy[b] * w3[k] : 0.f);
            dZ2[(int64_t)b * H + k] = v;
        }
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, b = b0 + threadIdx.x;
        if (k < H && b < B) dZ2T[(int64_t)k * B + b] = tile[threadIdx.x][r];
    }
}

// out[r] = sum_c M[r, c] (bf16 rows, fp32 sum), one warp per row.
__global__ void rowsum_kernel(const __nv_bfloat16 *Mx, int rows, int cols, float *out) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= rows) return;
    float s = 0.f;
    for (int c = lane; c < cols; c += 32) s += __bfloat162float(Mx[(int64_t)warp * cols + c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) out[warp] = s;
}

// dw3[k] = sum_b A2[b, k] dy[b]; db3 = sum_b dy[b] (thread k == H adds db3).
__global__ void dw3_kernel(const __nv_bfloat16 *A2, const float *dy, int B, int H, float *dw3, float *db3) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > H) return;
    float s = 0.f;
    if (k < H) {
        for (int b = 0; b < B; ++b) s = fmaf(__bfloat162float(A2[(int64_t)b * H + k]), dy[b], s);
        dw3[k] = s;
    } else {
        for (int b = 0; b < B; ++b) s += dy[b];
        db3[0] = s;
    }
}

// Adam on one tensor; writes the bf16 copy (and its transpose) if given.
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float c1, float c2, float eps, __nv_bfloat16 *pb, __nv_bfloat16 *pbt, int64_t rows,
                            int64_t cols) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = pi;
        if (pb) {
            const __nv_bfloat16 h = __float2bfloat16_rn(pi);
            pb[i] = h;
            if (pbt) pbt[(i % cols) * rows + i / cols] = h;
        }
    }
}

// Minibatch gather: row i = sample draw(u(seed, step, i), n_samples).
__global__ void gather_kernel(const int8_t *lv_all, const int64_t *ms_all, int64_t n_samples, int n_base, int B,
                              uint64_t seed, uint64_t step, int8_t *lv, int64_t *ms) {
    const int i = blockIdx.x;
    if (i >= B) return;
    const uint64_t u = sm64_at(seed, step, (uint64_t)i);
    const int64_t src = (int64_t)(((u >> 32) * (uint64_t)n_samples) >> 32);
    for (int t = threadIdx.x; t < n_base; t += blockDim.x) lv[(int64_t)i * n_base + t] = lv_all[src * n_base + t];
    if (threadIdx.x == 0) ms[i] = ms_all[src];
}

// mu, sigma of ln(makespan) over n samples (one block, deterministic order).
__global__ void stats_kernel(const int64_t *ms, int64_t n, double *out) {
    __shared__ double red[1024];
    double s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += log((double)ms[i]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double mu = red[0] / (double)n;
    __syncthreads();
    double q = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = log((double)ms[i]) - mu;
        q += d * d;
    }
    red[threadIdx.x] = q;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = mu;
        out[1] = sqrt(red[0] / (double)n);
    }
}

unsigned grid_for(int64_t n, int threads = 256) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int gemm(const void *A, int64_t lda, const void *Bm, int64_t ldb, int M, int N, int K, int epi, float *C, int ldc,
         const float *bias, __nv_bfloat16 *out, int ldo, __nv_bfloat16 *out_t, int ldt, const __nv_bfloat16 *mask,
         int ldm, int *err, cudaStream_t st) {
    GemmArgs g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = epi;
    g.C = C;
    g.ldc = ldc;
    g.bias = bias;
    g.out = out;
    g.ldo = ldo;
    g.out_t = out_t;
    g.ldt = ldt;
    g.mask = mask;
    g.ldm = ldm;
    g.err = err;
    return launch_gemm_bf16(A, lda, Bm, ldb, g, st);
}

#define CK(x)                                   \
    do {                                        \
        if ((x) != cudaSuccess) return HESP_ERR_CUDA; \
    } while (0)
#define RC(x)                 \
    do {                      \
        int rc_ = (x);        \
        if (rc_) return rc_;  \
    } while (0)

// Forward of B rows whose levels are at s->lv-like pointer `lv` (row stride
// n_base).  With ms != nullptr also the loss, dy and the backward pass.
int forward(hesp_surrogate *s, const int8_t *lv, int B, const int64_t *ms, float *pred, cudaStream_t st,
            bool backward) {
    const int H = s->H;
    const int64_t Fp = s->Fp;
    if (backward)
        onehot_t_kernel<<<grid_for((int64_t)Fp * (B / 8)), 256, 0, st>>>(lv, s->n_base, B, s->n_base, s->n_levels,
                                                                          (int)Fp, s->XT);
    CK(cudaGetLastError());
    {
        // layer 1: relu(onehot(levels) W1^T + b1), the one-hot operand built inside the GEMM
        GemmArgs g;
        g.M = B;
        g.N = H;
        g.K = (int)Fp;
        g.epi = 1;
        g.C = nullptr;
        g.ldc = 0;
        g.bias = s->b1;
        g.out = s->A1;
        g.ldo = H;
        g.out_t = backward ? s->A1T : nullptr;
        g.ldt = B;
        g.mask = nullptr;
        g.ldm = 0;
        g.err = s->err;
        const int8_t *lvg = lv;
        int64_t ld = s->n_base;
        if ((s->n_base & 15) || ((uintptr_t)lv & 15)) {
            pad_levels_kernel<<<grid_for((int64_t)B * s->n_base), 256, 0, st>>>(lv, s->n_base, B, (int)s->n_base,
                                                                                 (int)s->ldp, s->lvp);
            CK(cudaGetLastError());
            lvg = s->lvp;
            ld = s->ldp;
        }
        RC(launch_gemm_onehot(lvg, ld, (int)s->n_base, s->n_levels, s->W1b, Fp, g, st));
    }
    RC(gemm(s->A1, H, s->W2b, H, B, H, H, 1, nullptr, 0, s->b2, s->A2, H, nullptr, 0, nullptr, 0, s->err, st));
    l3_kernel<<<(unsigned)((B * 32 + 255) / 256), 256, 0, st>>>(s->A2, H, s->w3, s->b3, B, pred, ms, s->mu, s->sigma,
                                                               s->dy, s->sq);
    if (backward) loss_kernel<<<1, 1024, 0, st>>>(s->sq, B, s->loss);
    CK(cudaGetLastError());
    if (!backward) return HESP_OK;
    dz2_kernel<<<dim3((unsigned)((H + 31) / 32), (unsigned)((B + 31) / 32)), dim3(32, 8), 0, st>>>(
        s->A2, s->dy, s->w3, B, H, s->dZ2, s->dZ2T);
    CK(cudaGetLastError());
    dw3_kernel<<<(unsigned)((H + 1 + 127) / 128), 128, 0, st>>>(s->A2, s->dy, B, H, s->gw3, s->gb3);
    rowsum_kernel<<<(unsigned)((H * 32 + 255) / 256), 256, 0, st>>>(s->dZ2T, H, B, s->gb2);
    CK(cudaGetLastError());
    // dW2 = dZ2^T A1 (K = B)
    RC(gemm(s->dZ2T, B, s->A1T, B, H, H, B, 0, s->gW2, H, nullptr, nullptr, 0, nullptr, 0, nullptr, 0, s->err, st));
    // dZ1 = (dZ2 W2) * [A1 > 0]
    RC(gemm(s->dZ2, H, s->W2Tb, H, B, H, H, 2, nullptr, 0, nullptr, s->dZ1, H, s->dZ1T, B, s->A1, H, s->err, st));
    rowsum_kernel<<<(unsigned)((H * 32 + 255) / 256), 256, 0, st>>>(s->dZ1T, H, B, s->gb1);
    CK(cudaGetLastError());
    // dW1 = dZ1^T X (K = B)
    RC(gemm(s->dZ1T, B, s->XT, B, H, (int)Fp, B, 0, s->gW1, (int)Fp, nullptr, nullptr, 0, nullptr, 0, nullptr, 0,
            s->err, st));
    return HESP_OK;
}

int adam_all(hesp_surrogate *s, float lr, cudaStream_t st) {
    s->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, (double)s->step)));
    const float c2 = (float)(1.0 / (1.0 - pow(0.999, (double)s->step)));
    const int64_t H = s->H;
    struct T {
        float *p, *g, *m, *v;
        int64_t n;
        __nv_bfloat16 *pb, *pbt;
        int64_t rows, cols;
    } ts[6] = {{s->W1, s->gW1, s->mW1, s->vW1, H * s->Fp, s->W1b, nullptr, H, s->Fp},
               {s->b1, s->gb1, s->mb1, s->vb1, H, nullptr, nullptr, 1, H},
               {s->W2, s->gW2, s->mW2, s->vW2, H * H, s->W2b, s->W2Tb, H, H},
               {s->b2, s->gb2, s->mb2, s->vb2, H, nullptr, nullptr, 1, H},
               {s->w3, s->gw3, s->mw3, s->vw3, H, nullptr, nullptr, 1, H},
               {s->b3, s->gb3, s->mb3, s->vb3, 1, nullptr, nullptr, 1, 1}};
    for (auto &t : ts) {
        adam_kernel<<<grid_for(t.n), 256, 0, st>>>(t.p, t.g, t.m, t.v, t.n, lr, b1, b2, c1, c2, eps, t.pb, t.pbt,
                                                   t.rows, t.cols);
        CK(cudaGetLastError());
    }
    return HESP_OK;
}

int refresh_bf16(hesp_surrogate *s, cudaStream_t st) {
    const int64_t H = s->H;
    to_bf16_kernel<<<grid_for(H * s->Fp), 256, 0, st>>>(s->W1, s->W1b, nullptr, H, s->Fp);
    to_bf16_kernel<<<grid_for(H * H), 256, 0, st>>>(s->W2, s->W2b, s->W2Tb, H, H);
    CK(cudaGetLastError());
    return HESP_OK;
}

}  // namespace

extern "C" {

int hesp_surrogate_create(int32_t n_base, int32_t n_levels, int32_t hidden, int32_t max_batch, uint64_t seed,
                          hesp_surrogate **out) {
    if (!out) return HESP_ERR_ARG;
    *out = nullptr;
    if (n_base < 1 || n_levels < 1 || n_levels > HESP_MAX_LEVEL + 1 || hidden < 64 || hidden % 64 || max_batch < 64 ||
        max_batch % 64)
        return HESP_ERR_ARG;
    hesp_surrogate *s = (hesp_surrogate *)calloc(1, sizeof(hesp_surrogate));
    if (!s) return HESP_ERR_CAPACITY;
    s->n_base = n_base;
    s->n_levels = n_levels;
    s->H = hidden;
    s->max_batch = max_batch;
    s->F = (int64_t)n_base * n_levels;
    s->Fp = round_up(s->F, 64);
    s->seed = seed;
    s->mu = 0.0;
    s->sigma = 1.0;
    const int64_t H = hidden, Fp = s->Fp, B = max_batch;
    const int64_t nW1 = H * Fp, nW2 = H * H;
    // float block: 4 copies (p, g, m, v) of every tensor, each tensor starting
    // on a 256-byte boundary (vector stores in the GEMM epilogue need 16-byte
    // alignment), then y, dy, loss
    const int64_t sizes[6] = {nW1, H, nW2, H, H, 1};
    int64_t nparam = 0;
    for (int t = 0; t < 6; ++t) nparam += round_up(sizes[t], 64);
    size_t bytes = 0;
    auto take = [&](size_t n) {
        size_t o = bytes;
        bytes = (bytes + n + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_f = take(4 * (size_t)nparam * sizeof(float));
    const size_t o_y = take(B * sizeof(float));
    const size_t o_dy = take(B * sizeof(float)), o_sq = take(B * sizeof(float));
    const size_t o_loss = take(sizeof(float) + sizeof(int32_t) + 2 * sizeof(double));
    const size_t o_W1b = take(nW1 * 2), o_W2b = take(nW2 * 2), o_W2Tb = take(nW2 * 2);
    const size_t o_lv = take((size_t)B * n_base), o_ms = take(B * 8);
    const size_t o_XT = take((size_t)B * Fp * 2);
    s->ldp = round_up(n_base, 16);
    const size_t o_lvp = take((size_t)B * s->ldp);
    const size_t o_A1 = take(B * H * 2), o_A1T = take(B * H * 2), o_A2 = take(B * H * 2);
    const size_t o_dZ2 = take(B * H * 2), o_dZ2T = take(B * H * 2), o_dZ1 = take(B * H * 2),
                 o_dZ1T = take(B * H * 2);
    void *mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        free(s);
        return HESP_ERR_CUDA;
    }
    s->mem = mem;
    char *m = (char *)mem;
    float *f = (float *)(m + o_f);
    float **slots[4][6] = {{&s->W1, &s->b1, &s->W2, &s->b2, &s->w3, &s->b3},
                           {&s->gW1, &s->gb1, &s->gW2, &s->gb2, &s->gw3, &s->gb3},
                           {&s->mW1, &s->mb1, &s->mW2, &s->mb2, &s->mw3, &s->mb3},
                           {&s->vW1, &s->vb1, &s->vW2, &s->vb2, &s->vw3, &s->vb3}};
    for (int c = 0; c < 4; ++c)
        for (int t = 0; t < 6; ++t) {
            *slots[c][t] = f;
            f += round_up(sizes[t], 64);
        }
    s->y = (float *)(m + o_y);
    s->dy = (float *)(m + o_dy);
    s->loss = (float *)(m + o_loss);
    s->sq = (float *)(m + o_sq);
    s->err = (int32_t *)(m + o_loss + sizeof(float));
    s->W1b = (__nv_bfloat16 *)(m + o_W1b);
    s->W2b = (__nv_bfloat16 *)(m + o_W2b);
    s->W2Tb = (__nv_bfloat16 *)(m + o_W2Tb);
    s->lv = (int8_t *)(m + o_lv);
    s->ms = (int64_t *)(m + o_ms);
    s->XT = (__nv_bfloat16 *)(m + o_XT);
    s->lvp = (int8_t *)(m + o_lvp);
    s->A1 = (__nv_bfloat16 *)(m + o_A1);
    s->A1T = (__nv_bfloat16 *)(m + o_A1T);
    s->A2 = (__nv_bfloat16 *)(m + o_A2);
    s->dZ2 = (__nv_bfloat16 *)(m + o_dZ2);
    s->dZ2T = (__nv_bfloat16 *)(m + o_dZ2T);
    s->dZ1 = (__nv_bfloat16 *)(m + o_dZ1);
    s->dZ1T = (__nv_bfloat16 *)(m + o_dZ1T);
    if (cudaMemset(mem, 0, bytes) != cudaSuccess) return HESP_ERR_CUDA;
    const float bw1 = sqrtf(6.0f / (float)s->F), bw = sqrtf(6.0f / (float)H);
    init_uniform_kernel<<<grid_for(nW1), 256>>>(s->W1, H, Fp, s->F, seed, 0, bw1);
    init_uniform_kernel<<<grid_for(nW2), 256>>>(s->W2, H, H, H, seed, 1, bw);
    init_uniform_kernel<<<grid_for(H), 256>>>(s->w3, 1, H, H, seed, 2, bw);
    int rc = refresh_bf16(s, 0);
    if (rc || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(mem);
        free(s);
        return HESP_ERR_CUDA;
    }
    *out = s;
    return HESP_OK;
}

void hesp_surrogate_destroy(hesp_surrogate *s) {
    if (!s) return;
    cudaFree(s->mem);
    free(s);
}

int hesp_surrogate_shape(const hesp_surrogate *s, int64_t *F_out, int64_t *Fp_out, int32_t *H_out) {
    if (!s) return HESP_ERR_ARG;
    if (F_out) *F_out = s->F;
    if (Fp_out) *Fp_out = s->Fp;
    if (H_out) *H_out = s->H;
    return HESP_OK;
}

int hesp_surrogate_set_stats(hesp_surrogate *s, double mu, double sigma) {
    if (!s || !(sigma > 0)) return HESP_ERR_ARG;
    s->mu = mu;
    s->sigma = sigma;
    return HESP_OK;
}

int hesp_surrogate_get_stats(const hesp_surrogate *s, double *mu, double *sigma, int64_t *step) {
    if (!s) return HESP_ERR_ARG;
    if (mu) *mu = s->mu;
    if (sigma) *sigma = s->sigma;
    if (step) *step = s->step;
    return HESP_OK;
}

int hesp_surrogate_fit_stats(hesp_surrogate *s, const int64_t *makespan_dev, int64_t n, void *stream) {
    if (!s || !makespan_dev || n < 1) return HESP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *d = (double *)((char *)s->loss + 8);
    stats_kernel<<<1, 1024, 0, st>>>(makespan_dev, n, d);
    double h[2];
    if (cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return HESP_ERR_CUDA;
    if (!(h[1] > 0)) return HESP_ERR_ARG;
    s->mu = h[0];
    s->sigma = h[1];
    return HESP_OK;
}

// Parameter / gradient / moment transfer through host buffers, in the order
// W1 [H, Fp], b1 [H], W2 [H, H], b2 [H], w3 [H], b3 [1] (fp32, contiguous).
// which: 0 parameters, 1 gradients, 2 first moments, 3 second moments.
static int tensor_list(const hesp_surrogate *s, int which, float *ptrs[6], int64_t sizes[6]) {
    const int64_t H = s->H;
    float *const all[4][6] = {{s->W1, s->b1, s->W2, s->b2, s->w3, s->b3},
                              {s->gW1, s->gb1, s->gW2, s->gb2, s->gw3, s->gb3},
                              {s->mW1, s->mb1, s->mW2, s->mb2, s->mw3, s->mb3},
                              {s->vW1, s->vb1, s->vW2, s->vb2, s->vw3, s->vb3}};
    const int64_t sz[6] = {H * s->Fp, H, H * H, H, H, 1};
    for (int t = 0; t < 6; ++t) {
        ptrs[t] = all[which][t];
        sizes[t] = sz[t];
    }
    return HESP_OK;
}

int hesp_surrogate_get(const hesp_surrogate *s, int32_t which, float *host, int64_t n) {
    if (!s || !host || which < 0 || which > 3) return HESP_ERR_ARG;
    float *ptrs[6];
    int64_t sizes[6];
    tensor_list(s, which, ptrs, sizes);
    int64_t tot = 0;
    for (int t = 0; t < 6; ++t) tot += sizes[t];
    if (n != tot) return HESP_ERR_ARG;
    for (int t = 0; t < 6; ++t) {
        if (cudaMemcpy(host, ptrs[t], sizes[t] * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
            return HESP_ERR_CUDA;
        host += sizes[t];
    }
    return HESP_OK;
}

int hesp_surrogate_set(hesp_surrogate *s, int32_t which, const float *host, int64_t n) {
    if (!s || !host || which < 0 || which > 3) return HESP_ERR_ARG;
    float *ptrs[6];
    int64_t sizes[6];
    tensor_list(s, which, ptrs, sizes);
    int64_t tot = 0;
    for (int t = 0; t < 6; ++t) tot += sizes[t];
    if (n != tot) return HESP_ERR_ARG;
    for (int t = 0; t < 6; ++t) {
        if (cudaMemcpy(ptrs[t], host, sizes[t] * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return HESP_ERR_CUDA;
        host += sizes[t];
    }
    if (which == 0) {
        const int rc = refresh_bf16(s, 0);
        if (rc) return rc;
        if (cudaDeviceSynchronize() != cudaSuccess) return HESP_ERR_CUDA;
    }
    return HESP_OK;
}

// Forward + backward on a given batch (levels_dev [B, n_base], makespan_dev
// [B]); gradients land in the gradient buffers, the loss in *loss_dev and
// the predictions in pred_dev (both nullable).  No parameter update.
int hesp_surrogate_grad(hesp_surrogate *s, const int8_t *levels_dev, const int64_t *makespan_dev, int32_t B,
                        float *pred_dev, float *loss_dev, void *stream) {
    if (!s || !levels_dev || !makespan_dev || B < 64 || B % 64 || B > s->max_batch) return HESP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    RC(forward(s, levels_dev, B, makespan_dev, s->y, st, true));
    if (pred_dev) CK(cudaMemcpyAsync(pred_dev, s->y, B * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (loss_dev) CK(cudaMemcpyAsync(loss_dev, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
    return HESP_OK;
}

// Apply one Adam step to the gradients currently held (learning rate lr).
int hesp_surrogate_adam(hesp_surrogate *s, float lr, void *stream) {
    if (!s || !(lr >= 0)) return HESP_ERR_ARG;
    return adam_all(s, lr, (cudaStream_t)stream);
}

// n_steps Adam steps on minibatches of `batch` rows drawn (SplitMix64, seeded
// by `seed` and the step number) from the n_samples labelled samples.
// loss_dev (nullable) receives the loss of every step [n_steps].
int hesp_surrogate_train(hesp_surrogate *s, const int8_t *levels_dev, const int64_t *makespan_dev, int64_t n_samples,
                         int32_t batch, int32_t n_steps, float lr, uint64_t seed, float *loss_dev, void *stream) {
    if (!s || !levels_dev || !makespan_dev || n_samples < 1 || batch < 64 || batch % 64 || batch > s->max_batch ||
        n_steps < 0 || !(lr >= 0))
        return HESP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    for (int k = 0; k < n_steps; ++k) {
        gather_kernel<<<batch, 128, 0, st>>>(levels_dev, makespan_dev, n_samples, s->n_base, batch, seed,
                                              (uint64_t)(s->step), s->lv, s->ms);
        CK(cudaGetLastError());
        RC(forward(s, s->lv, batch, s->ms, s->y, st, true));
        if (loss_dev) CK(cudaMemcpyAsync(loss_dev + k, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
        RC(adam_all(s, lr, st));
    }
    return HESP_OK;
}

// Predicted standardised log-makespan of n candidates (levels_dev [n, n_base]).
int hesp_surrogate_infer(hesp_surrogate *s, const int8_t *levels_dev, int64_t n, float *pred_dev, void *stream) {
    if (!s || !levels_dev || !pred_dev || n < 0) return HESP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t i = 0; i < n; i += s->max_batch) {
        const int B = (int)((n - i) < s->max_batch ? (n - i) : s->max_batch);
        RC(forward(s, levels_dev + i * s->n_base, B, nullptr, pred_dev + i, st, false));
    }
    return HESP_OK;
}

int hesp_surrogate_error(hesp_surrogate *s, int32_t *err_host) {
    if (!s || !err_host) return HESP_ERR_ARG;
    return cudaMemcpy(err_host, s->err, sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess ? HESP_OK
                                                                                              : HESP_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoints
// File layout, little-endian: the 8 bytes "HESPSUR1"; int32 n_base,
// n_levels, H, max_batch; uint64 seed; int64 step; float64 mu, sigma; int64
// F, Fp; then the six FP32 tensors (W1, b1, W2, b2, w3, b3) of the
// parameters, of the Adam first moments and of the second moments; then the
// 64-bit FNV-1a hash of every byte before it.

namespace {

constexpr char kMagic[8] = {'H', 'E', 'S', 'P', 'S', 'U', 'R', '1'};

struct CkptHeader {
    char magic[8];
    int32_t n_base, n_levels, H, max_batch;
    uint64_t seed;
    int64_t step;
    double mu, sigma;
    int64_t F, Fp;
};

uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

int64_t ckpt_floats(const hesp_surrogate *s) {
    float *ptrs[6];
    int64_t sizes[6];
    tensor_list(s, 0, ptrs, sizes);
    int64_t tot = 0;
    for (int t = 0; t < 6; ++t) tot += sizes[t];
    return tot;
}

}  // namespace

int hesp_surrogate_save(const hesp_surrogate *s, const char *path) {
    if (!s || !path) return HESP_ERR_ARG;
    CkptHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, kMagic, 8);
    hd.n_base = s->n_base;
    hd.n_levels = s->n_levels;
    hd.H = s->H;
    hd.max_batch = s->max_batch;
    hd.seed = s->seed;
    hd.step = s->step;
    hd.mu = s->mu;
    hd.sigma = s->sigma;
    hd.F = s->F;
    hd.Fp = s->Fp;
    const int64_t nf = ckpt_floats(s);
    float *buf = (float *)malloc((size_t)nf * sizeof(float));
    if (!buf) return HESP_ERR_CAPACITY;
    char *tmp = (char *)malloc(strlen(path) + 8);
    if (!tmp) {
        free(buf);
        return HESP_ERR_CAPACITY;
    }
    sprintf(tmp, "%s.tmp", path);
    FILE *f = fopen(tmp, "wb");
    int rc = f ? HESP_OK : HESP_ERR_ARG;
    uint64_t h = 0xcbf29ce484222325ull;
    if (rc == HESP_OK) {
        h = fnv1a(h, &hd, sizeof hd);
        if (fwrite(&hd, sizeof hd, 1, f) != 1) rc = HESP_ERR_ARG;
    }
    const int which[3] = {0, 2, 3};
    for (int k = 0; k < 3 && rc == HESP_OK; ++k) {
        rc = hesp_surrogate_get(s, which[k], buf, nf);
        if (rc) break;
        h = fnv1a(h, buf, (size_t)nf * sizeof(float));
        if (fwrite(buf, sizeof(float), (size_t)nf, f) != (size_t)nf) rc = HESP_ERR_ARG;
    }
    if (rc == HESP_OK && fwrite(&h, sizeof h, 1, f) != 1) rc = HESP_ERR_ARG;
    if (f && fclose(f) != 0 && rc == HESP_OK) rc = HESP_ERR_ARG;
    if (rc == HESP_OK && rename(tmp, path) != 0) rc = HESP_ERR_ARG;
    if (rc != HESP_OK) remove(tmp);
    free(tmp);
    free(buf);
    return rc;
}

int hesp_surrogate_load(const char *path, hesp_surrogate **out) {
    if (!path || !out) return HESP_ERR_ARG;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return HESP_ERR_ARG;
    CkptHeader hd;
    if (fread(&hd, sizeof hd, 1, f) != 1 || memcmp(hd.magic, kMagic, 8) != 0) {
        fclose(f);
        return HESP_ERR_ARG;
    }
    hesp_surrogate *s = nullptr;
    int rc = hesp_surrogate_create(hd.n_base, hd.n_levels, hd.H, hd.max_batch, hd.seed, &s);
    if (rc) {
        fclose(f);
        return rc;
    }
    if (s->F != hd.F || s->Fp != hd.Fp || !(hd.sigma > 0) || hd.step < 0) rc = HESP_ERR_ARG;
    const int64_t nf = ckpt_floats(s);
    float *buf[3] = {nullptr, nullptr, nullptr};
    uint64_t h = fnv1a(0xcbf29ce484222325ull, &hd, sizeof hd);
    for (int k = 0; k < 3 && rc == HESP_OK; ++k) {
        buf[k] = (float *)malloc((size_t)nf * sizeof(float));
        if (!buf[k]) rc = HESP_ERR_CAPACITY;
        else if (fread(buf[k], sizeof(float), (size_t)nf, f) != (size_t)nf) rc = HESP_ERR_ARG;
        else h = fnv1a(h, buf[k], (size_t)nf * sizeof(float));
    }
    uint64_t want = 0;
    if (rc == HESP_OK && (fread(&want, sizeof want, 1, f) != 1 || want != h)) rc = HESP_ERR_ARG;
    if (rc == HESP_OK && fgetc(f) != EOF) rc = HESP_ERR_ARG;  // trailing bytes
    fclose(f);
    const int which[3] = {0, 2, 3};
    for (int k = 0; k < 3 && rc == HESP_OK; ++k) rc = hesp_surrogate_set(s, which[k], buf[k], nf);
    for (int k = 0; k < 3; ++k) free(buf[k]);
    if (rc == HESP_OK) {
        s->step = hd.step;
        s->mu = hd.mu;
        s->sigma = hd.sigma;
        *out = s;
    } else {
        hesp_surrogate_destroy(s);
    }
    return rc;
}
