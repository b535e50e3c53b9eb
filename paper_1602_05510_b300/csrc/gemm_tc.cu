// BF16 tensor-core GEMM for sm_103a (5th-generation tensor cores):
//     C[M, N] = A[M, K] . B[N, K]^T      (A, B bf16, K contiguous; FP32 accumulate)
// with fused epilogues for the surrogate MLP's layers.
//
// One CTA computes a 128 x 128 tile of C.  Warp 0 (one elected lane) streams
// 128 x 64 tiles of A and B into a 3-stage shared-memory ring with TMA
// (cp.async.bulk.tensor, 128-byte swizzle); warp 1 (one lane) issues
// tcgen05.mma (M = 128, N = 128, K = 16 per instruction) into a TMEM
// accumulator and releases each stage with tcgen05.commit on its "empty"
// mbarrier; warp 2 owns the TMEM allocation; all four warps then drain the
// accumulator with tcgen05.ld (warp w reads TMEM lanes 32w .. 32w+31 = rows)
// and apply the epilogue.  Two CTAs fit one SM (~100 KB of shared memory and
// 128 TMEM columns each), so one CTA's epilogue overlaps the other's main
// loop.  Every mbarrier wait is bounded: on expiry the CTA
// raises the caller's error flag, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "hesp_internal.h"

namespace hesp {


namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 2;  // 16 KiB per operand per stage
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(a, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm, uint32_t mbar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"((uint64_t)tm), "r"(mbar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand tile, rows of 64 bf16
// (128 bytes) with the 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride-dimension offset: next 8-row group
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor: dense, D = f32, A = B = bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(128, 2)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint32_t *holder = (uint32_t *)(bars + 2 * STAGES + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int KT = g.K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;

    bool fail = false;
    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kt = 0; kt < KT; ++kt) {
            const int s = kt % STAGES;
            if (kt >= STAGES && !mbar_wait(empty0 + 8 * s, ((kt / STAGES) - 1) & 1)) {
                fail = true;
                break;
            }
            mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
            tma_load_2d(sa, &tmA, full0 + 8 * s, kt * BK, m0);
            tma_load_2d(sa + TILE_BYTES, &tmB, full0 + 8 * s, kt * BK, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BM, BN);
        for (int kt = 0; kt < KT; ++kt) {
            const int s = kt % STAGES;
            if (!mbar_wait(full0 + 8 * s, (kt / STAGES) & 1)) {
                fail = true;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t da = sw128_desc(sa + kk * 32);
                const uint64_t db = sw128_desc(sa + TILE_BYTES + kk * 32);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 +
                                                                                                           8 * s)
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                     : "memory");
    }
    __syncwarp();
    const bool ready = __all_sync(0xFFFFFFFFu, !fail && mbar_wait(done, 0));
    tc_fence_after();
    if (ready) {
        const int row = m0 + warp * 32 + lane;
        const bool rok = row < g.M;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            const int col0 = n0 + c0;
            if (!rok || col0 >= g.N) continue;
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
            const bool full = col0 + 16 <= g.N;
            if (g.epi == 0) {
                float *dst = g.C + (int64_t)row * g.ldc + col0;
                if (full && (((uintptr_t)dst) & 15) == 0) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4) *reinterpret_cast<float4 *>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                } else {
                    for (int q = 0; q < 16 && col0 + q < g.N; ++q) dst[q] = v[q];
                }
                continue;
            }
            if (g.epi == 1) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float bq = (col0 + q < g.N) ? g.bias[col0 + q] : 0.f;
                    v[q] = fmaxf(v[q] + bq, 0.f);
                }
            } else {
                const __nv_bfloat16 *mk = g.mask + (int64_t)row * g.ldm + col0;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (col0 + q < g.N && !(__bfloat162float(mk[q]) > 0.f)) v[q] = 0.f;
            }
            __nv_bfloat16 h[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) h[q] = __float2bfloat16_rn(v[q]);
            __nv_bfloat16 *dst = g.out + (int64_t)row * g.ldo + col0;
            if (full && (((uintptr_t)dst) & 15) == 0) {
                *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(h);
                *reinterpret_cast<uint4 *>(dst + 8) = *reinterpret_cast<const uint4 *>(h + 8);
            } else {
                for (int q = 0; q < 16 && col0 + q < g.N; ++q) dst[q] = h[q];
            }
            if (g.out_t) {
                for (int q = 0; q < 16 && col0 + q < g.N; ++q) g.out_t[(int64_t)(col0 + q) * g.ldt + row] = h[q];
            }
        }
    }
    if ((fail || !ready) && g.err && lane == 0) atomicExch(g.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

int get_encode() {
    std::lock_guard<std::mutex> lk(g_encode_mu);
    if (g_encode) return HESP_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return HESP_ERR_CUDA;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return HESP_OK;
}

// Tensor map of a row-major bf16 matrix [rows, ld] read in 128 x 64 boxes.
int make_map(CUtensorMap *tm, const void *ptr, int64_t rows, int64_t cols, int64_t ld) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {BK, BM};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HESP_OK : HESP_ERR_ARG;
}

}  // namespace

// C = A . B^T; A [M, lda] and B [N, ldb] bf16 with K (multiple of 64) used
// columns; lda, ldb multiples of 8; base addresses 16-byte aligned.
int launch_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, const GemmArgs &g, cudaStream_t st) {
    if (g.M < 1 || g.N < 1 || g.K < BK || g.K % BK || (lda & 7) || (ldb & 7) || lda < g.K || ldb < g.K)
        return HESP_ERR_ARG;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return HESP_ERR_ARG;
    int rc = get_encode();
    if (rc) return rc;
    CUtensorMap ta, tb;
    if ((rc = make_map(&ta, A, g.M, g.K, lda))) return rc;
    if ((rc = make_map(&tb, B, g.N, g.K, ldb))) return rc;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
            cudaSuccess)
            return HESP_ERR_CUDA;
        attr_set = true;
    }
    dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM));
    gemm_bf16_kernel<<<grid, 128, SMEM_BYTES, st>>>(ta, tb, g);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

}  // namespace hesp

using namespace hesp;

extern "C" int hesp_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *a_dev, int64_t lda, const void *b_dev,
                              int64_t ldb, int32_t epilogue, float *c_dev, int64_t ldc, const float *bias_dev,
                              void *out_dev, int64_t ldo, void *out_t_dev, int64_t ldt, const void *mask_dev,
                              int64_t ldm, int32_t *err_dev, void *stream) {
    if (!a_dev || !b_dev || epilogue < 0 || epilogue > 2) return HESP_ERR_ARG;
    if (epilogue == 0 && (!c_dev || ldc < N)) return HESP_ERR_ARG;
    if (epilogue == 1 && (!bias_dev || !out_dev || ldo < N)) return HESP_ERR_ARG;
    if (epilogue == 2 && (!mask_dev || !out_dev || ldo < N || ldm < N)) return HESP_ERR_ARG;
    if (out_t_dev && ldt < M) return HESP_ERR_ARG;
    GemmArgs g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = epilogue;
    g.C = c_dev;
    g.ldc = (int)ldc;
    g.bias = bias_dev;
    g.out = (__nv_bfloat16 *)out_dev;
    g.ldo = (int)ldo;
    g.out_t = (__nv_bfloat16 *)out_t_dev;
    g.ldt = (int)ldt;
    g.mask = (const __nv_bfloat16 *)mask_dev;
    g.ldm = (int)ldm;
    g.err = err_dev;
    return launch_gemm_bf16(a_dev, lda, b_dev, ldb, g, (cudaStream_t)stream);
}
