// BF16 tensor-core GEMM for sm_103a (5th-generation tensor cores):
//     C[M, N] = A[M, K] . B[N, K]^T      (A, B bf16, K contiguous; FP32 accumulate)
// with fused epilogues for the surrogate MLP's layers.
//
// Persistent and warp-specialised, one CTA per SM: each CTA walks 128 x 256
// output tiles (blockIdx.x, + gridDim.x, ...; the N-tiles of one row block
// are consecutive).  Warp 0 (one lane) streams 64-column k-blocks of B (256
// rows) -- and of A (128 rows), unless A is built in place -- into a 4-stage
// shared-memory ring with TMA (cp.async.bulk.tensor, 128-byte swizzle); warp 1
// (one lane) issues tcgen05.mma (M = 128, N = 256, K = 16 per instruction)
// into one of two TMEM accumulators (2 x 256 columns, all of TMEM) and frees
// each stage with tcgen05.commit; warps 2-9 drain the other accumulator
// (tcgen05.ld; warp w reads TMEM lanes 32 (w % 4) .. + 31, warps 2-5 the first
// 128 columns and 6-9 the last) and apply the epilogue, so a tile's epilogue
// runs under the next tile's main loop.
//
// With NL > 0 the A operand is the one-hot encoding of int8 levels,
// X[r, f] = (levels[r, f / NL] == f % NL) for f < n_base NL (else 0), and
// warps 10-17 build its tiles in shared memory (two groups of four taking
// alternate k-blocks; thread r of a group writes row r, eight 16-byte chunks
// per k-block, in the same swizzled layout) from level windows that TMA
// brings with B, so the one-hot matrix never exists in memory.  A chunk of
// 8 features starting at phase v0 = f % NL spans at most S tasks; its 16
// bytes are read from a table, built once per CTA, indexed by (v0, the S
// levels).
//
// Every mbarrier wait is bounded: on expiry the role stops, the caller's error
// flag is raised, and the CTA frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "hesp_internal.h"

namespace hesp {


namespace {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int A_BYTES = BM * BK * 2;  // 16 KiB
constexpr int B_BYTES = BN * BK * 2;  // 32 KiB
constexpr int SMEM_LIMIT = 227 * 1024;  // dynamic shared memory of one CTA

constexpr int TMEM_COLS = 2 * BN;  // two accumulators: all of TMEM, one CTA per SM
constexpr int N_EPI_WARPS = 8;
constexpr uint32_t kWaitLimit = 1u << 22;

// tasks spanned by 8 consecutive features, at most, for NL levels per task
__host__ __device__ constexpr int span_of(int nl) { return nl <= 0 ? 1 : (nl - 1 + 8 + nl - 1) / nl; }
__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
// level bytes a 64-feature k-block reads (the S tasks from each chunk's first
// task), in 32-bit words
__host__ __device__ constexpr int window_words(int nl) { return ((nl - 1 + 56) / nl + span_of(nl) + 3) / 4; }
// Per instantiation (NL = 0: TMA A operand; NL > 0: A built from levels):
// the level box width (its start is rounded down to 16 bytes, and the window
// is read as window_words + 1 words from a 4-byte boundary), the chunk
// table, the stage size and as many stages (3 or 4) as shared memory holds.
__host__ __device__ constexpr int lv_cols_of(int nl) {
    return nl == 0 ? 0 : (12 + 4 * (window_words(nl) + 1) + 15) / 16 * 16;
}
__host__ __device__ constexpr int table_bytes_of(int nl) {
    return nl == 0 ? 0 : (nl * ipow(nl, span_of(nl)) * 16 + 127) / 128 * 128;
}
__host__ __device__ constexpr int stage_bytes_of(int nl) { return A_BYTES + B_BYTES + BM * lv_cols_of(nl); }
__host__ __device__ constexpr int smem_for(int nl, int stages) {
    return 1024 + stages * stage_bytes_of(nl) + table_bytes_of(nl) + 512;
}
__host__ __device__ constexpr int stages_of(int nl) { return smem_for(nl, 4) <= SMEM_LIMIT ? 4 : 3; }
__host__ __device__ constexpr int smem_bytes_of(int nl) { return smem_for(nl, stages_of(nl)); }
static_assert(stage_bytes_of(1) % 1024 == 0 && stage_bytes_of(2) % 1024 == 0 && stage_bytes_of(3) % 1024 == 0 &&
                  stage_bytes_of(4) % 1024 == 0 && stage_bytes_of(5) % 1024 == 0,
              "stages must keep the 128-byte-swizzled tiles 1024-byte aligned");
static_assert(smem_bytes_of(0) <= SMEM_LIMIT && smem_bytes_of(1) <= SMEM_LIMIT && smem_bytes_of(5) <= SMEM_LIMIT,
              "shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
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

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes; the
// caller waits (tmem_wait) before reading r.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// bf16 bits of x, round to nearest even
__device__ __forceinline__ uint32_t bf16_bits(float x) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// Epilogue of 16 accumulator columns of one output row.  Every index is a
// compile-time constant, so the values stay in registers.
__device__ __forceinline__ void epilogue16(const GemmArgs &g, int row, int col0, const uint32_t (&r)[16]) {
    float v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
    const bool full = col0 + 16 <= g.N;
    if (g.epi == 0) {
        float *dst = g.C + (int64_t)row * g.ldc + col0;
        if (full && (((uintptr_t)dst) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < 16; q += 4)
                *reinterpret_cast<float4 *>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (col0 + q < g.N) dst[q] = v[q];
        }
        return;
    }
    if (g.epi == 1) {
        const float *bp = g.bias + col0;
        if (full && (((uintptr_t)bp) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < 16; q += 4) {
                const float4 b4 = __ldg(reinterpret_cast<const float4 *>(bp + q));
                v[q] = fmaxf(v[q] + b4.x, 0.f);
                v[q + 1] = fmaxf(v[q + 1] + b4.y, 0.f);
                v[q + 2] = fmaxf(v[q + 2] + b4.z, 0.f);
                v[q + 3] = fmaxf(v[q + 3] + b4.w, 0.f);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float bq = (col0 + q < g.N) ? bp[q] : 0.f;
                v[q] = fmaxf(v[q] + bq, 0.f);
            }
        }
    } else {
        const __nv_bfloat16 *mk = g.mask + (int64_t)row * g.ldm + col0;
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (col0 + q < g.N && !(__bfloat162float(mk[q]) > 0.f)) v[q] = 0.f;
    }
    uint32_t w[8];  // bf16 pairs
#pragma unroll
    for (int q = 0; q < 8; ++q) w[q] = bf16_bits(v[2 * q]) | (bf16_bits(v[2 * q + 1]) << 16);
    __nv_bfloat16 *dst = g.out + (int64_t)row * g.ldo + col0;
    if (full && (((uintptr_t)dst) & 15) == 0) {
        *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(dst + 8) = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (col0 + q < g.N) dst[q] = __ushort_as_bfloat16((unsigned short)(w[q >> 1] >> (16 * (q & 1))));
    }
    if (g.out_t) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (col0 + q < g.N)
                g.out_t[(int64_t)(col0 + q) * g.ldt + row] =
                    __ushort_as_bfloat16((unsigned short)(w[q >> 1] >> (16 * (q & 1))));
    }
}

// One 64-feature k-block of one one-hot row, whose first feature has phase V
// (= f % NL) and whose tasks start at window byte 0 (n_valid of the window's
// bytes are tasks of the row).  Chunk c covers features V + 8c .. + 7 of the
// window: tasks i0 = (V + 8c) / NL .. i0 + S - 1, phase v0 = (V + 8c) % NL.
// With the whole window valid (tasks of the row, levels < NL) a chunk is one
// table entry; otherwise each feature is compared on its own (bf16 1.0 where
// the level matches, 0 past the row or for an invalid level).
template <int NL, int V, int WW>
__device__ __forceinline__ void onehot_kblock(const uint32_t (&w)[WW], const uint4 *table, uint8_t *arow, int r,
                                              int n_valid) {
    constexpr int S = span_of(NL);
    uint32_t bad = n_valid < 4 * WW ? 1u : 0u;  // the window runs past the row's last task
#pragma unroll
    for (int i = 0; i < WW; ++i)  // a byte >= NL: bit 7 set, or bit 7 after adding 128 - NL to its low 7 bits
        bad |= (w[i] | ((w[i] & 0x7F7F7F7Fu) + (uint32_t)(128 - NL) * 0x01010101u)) & 0x80808080u;
    if (bad == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int p = V + 8 * c;
            const int i0 = p / NL, v0 = p % NL;
            int idx = v0;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const int bi = i0 + i;
                idx = idx * NL + (int)((w[bi >> 2] >> (8 * (bi & 3))) & 0xFFu);
            }
            *reinterpret_cast<uint4 *>(arow + ((c ^ (r & 7)) << 4)) = table[idx];
        }
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t o[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int p0 = V + 8 * c + 2 * h, p1 = p0 + 1;
                const int b0 = p0 / NL, b1 = p1 / NL;
                const uint32_t l0 = b0 < n_valid ? (w[b0 >> 2] >> (8 * (b0 & 3))) & 0xFFu : 0xFFu;
                const uint32_t l1 = b1 < n_valid ? (w[b1 >> 2] >> (8 * (b1 & 3))) & 0xFFu : 0xFFu;
                o[h] = (l0 == (uint32_t)(p0 % NL) ? 0x3F80u : 0u) | ((l1 == (uint32_t)(p1 % NL) ? 0x3F80u : 0u) << 16);
            }
            *reinterpret_cast<uint4 *>(arow + ((c ^ (r & 7)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
        }
    }
}

constexpr int N_PROD_GROUPS = 2;  // A-producer groups of 4 warps, taking alternate k-blocks

template <int NL>
__global__ void __launch_bounds__(NL > 0 ? 320 + 128 * N_PROD_GROUPS : 320, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmL, GemmArgs g) {
    constexpr int STAGES = stages_of(NL), STAGE_BYTES = stage_bytes_of(NL);
    constexpr int NBARS = 3 * STAGES + 4;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint4 *table = (uint4 *)(smem + STAGES * STAGE_BYTES);
    uint64_t *bars = (uint64_t *)(smem + STAGES * STAGE_BYTES + table_bytes_of(NL));
    uint32_t *holder = (uint32_t *)(bars + NBARS);
    // full: the stage is ready for the MMA; empty: the MMA is done with it;
    // lfull (NL > 0): B and the level window have landed; tfull / tempty: an
    // accumulator is complete / drained
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), lfull0 = smem_u32(bars + 2 * STAGES);
    const uint32_t tfull0 = smem_u32(bars + 3 * STAGES), tempty0 = smem_u32(bars + 3 * STAGES + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int KT = g.K / BK;
    const int nN = (g.N + BN - 1) / BN;
    const int n_tiles = ((g.M + BM - 1) / BM) * nN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, NL > 0 ? 4 : 1);  // one lane per warp of the producer group, or the TMA thread
            mbar_init(empty0 + 8 * s, 1);
            mbar_init(lfull0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, N_EPI_WARPS);  // one lane per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;

    bool fail = false;
    if (warp == 0) {
        if (lane == 0) {
            // TMA producer: A and B (NL = 0), or B and the level window (NL > 0)
            int it = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !fail; tile += gridDim.x) {
                const int m0 = (tile / nN) * BM, n0 = (tile % nN) * BN;
                for (int kt = 0; kt < KT; ++kt, ++it) {
                    const int s = it % STAGES, q = it / STAGES;
                    if (q > 0 && !mbar_wait(empty0 + 8 * s, (q - 1) & 1)) {
                        fail = true;
                        break;
                    }
                    const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                    if constexpr (NL == 0) {
                        mbar_expect_tx(full0 + 8 * s, A_BYTES + B_BYTES);
                        tma_load_2d(sa, &tmA, full0 + 8 * s, kt * BK, m0);
                        tma_load_2d(sa + A_BYTES, &tmB, full0 + 8 * s, kt * BK, n0);
                    } else {
                        // tasks from t_kb on; the box starts at t_kb rounded down to 16 bytes
                        const int t_kb = (kt * BK) / NL;
                        mbar_expect_tx(lfull0 + 8 * s, B_BYTES + BM * lv_cols_of(NL));
                        tma_load_2d(sa + A_BYTES, &tmB, lfull0 + 8 * s, kt * BK, n0);
                        tma_load_2d(sa + A_BYTES + B_BYTES, &tmL, lfull0 + 8 * s, t_kb & ~15, m0);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            int it = 0, i = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !fail; tile += gridDim.x, ++i) {
                const int acc_i = i & 1, use = i >> 1;
                if (use > 0 && !mbar_wait(tempty0 + 8 * acc_i, (use - 1) & 1)) {
                    fail = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc_i * BN);
                for (int kt = 0; kt < KT; ++kt, ++it) {
                    const int s = it % STAGES, q = it / STAGES;
                    if (!mbar_wait(full0 + 8 * s, q & 1)) {
                        fail = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t da = sw128_desc(sa + kk * 32);
                        const uint64_t db = sw128_desc(sa + A_BYTES + kk * 32);
                        const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\t"
                            "setp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                            "l"(da), "l"(db), "r"(idesc), "r"(accum)
                            : "memory");
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 +
                                                                                                            8 * s)
                        : "memory");
                }
                if (fail) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tfull0 + 8 * acc_i)
                             : "memory");
            }
        }
    } else if (warp < 2 + N_EPI_WARPS) {
        // epilogue: rows 32 (warp % 4) .. + 31 of each tile, columns
        // 128 h .. + 127 with h = (warp - 2) / 4
        const int wq = warp & 3, h = (warp - 2) >> 2;
        int i = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
            const int acc_i = i & 1, use = i >> 1;
            const bool ok = __all_sync(0xFFFFFFFFu, mbar_wait(tfull0 + 8 * acc_i, use & 1));
            if (!ok) {
                fail = true;
                break;
            }
            tc_fence_after();
            const int m0 = (tile / nN) * BM, n0 = (tile % nN) * BN;
            const int row = m0 + wq * 32 + lane;
            const bool rok = row < g.M;
            const uint32_t tbase = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(acc_i * BN);
            for (int c0 = h * 128; c0 < h * 128 + 128; c0 += 32) {  // two loads in flight per wait
                uint32_t r0[16], r1[16];
                tmem_ld16(tbase + (uint32_t)c0, r0);
                tmem_ld16(tbase + (uint32_t)(c0 + 16), r1);
                tmem_wait();
                if (rok && n0 + c0 < g.N) epilogue16(g, row, n0 + c0, r0);
                if (rok && n0 + c0 + 16 < g.N) epilogue16(g, row, n0 + c0 + 16, r1);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * acc_i);
        }
    } else if constexpr (NL > 0) {
        // A producers (warps 10 on, two groups of four taking alternate
        // k-blocks): the chunk table, then for each of the group's k-blocks,
        // once B and the level window have landed, thread r of the group
        // builds row r of the A tile from its window, with byte positions
        // fixed by the k-block's phase.  The only barrier across the producer
        // warps is the one after the table is built, before any wait that can
        // time out.
        constexpr int S = span_of(NL);
        constexpr int NE = NL * ipow(NL, S);
        constexpr int WW = window_words(NL);
        const int ptid = threadIdx.x - 32 * (2 + N_EPI_WARPS);
        const int grp = ptid >> 7, tid = ptid & 127;
        for (int e = ptid; e < NE; e += 128 * N_PROD_GROUPS) {
            int rem = e, lv_[S];
#pragma unroll
            for (int i = S - 1; i >= 0; --i) {
                lv_[i] = rem % NL;
                rem /= NL;
            }
            const int v0 = rem;
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                const int p0 = v0 + q, p1 = v0 + q + 1;
                const uint32_t lo = lv_[p0 / NL] == p0 % NL ? 0x3F80u : 0u;
                const uint32_t hi = lv_[p1 / NL] == p1 % NL ? 0x3F80u : 0u;
                w[q >> 1] = lo | (hi << 16);
            }
            table[e] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(128 * N_PROD_GROUPS) : "memory");  // the producer warps
        const int r = tid;
        const int nb = g.oh_base;
        int it = 0;
        for (int tile = blockIdx.x; tile < n_tiles && !fail; tile += gridDim.x) {
            for (int kt = 0; kt < KT; ++kt, ++it) {
                if ((it % N_PROD_GROUPS) != grp) continue;
                const int s = it % STAGES, q = it / STAGES;
                if (!__all_sync(0xFFFFFFFFu, mbar_wait(lfull0 + 8 * s, q & 1))) {
                    fail = true;
                    break;
                }
                const int t_kb = (kt * BK) / NL, v_kb = kt * BK - t_kb * NL;
                const int o = t_kb & 15;  // window start inside the 16-byte aligned box
                const uint32_t *lrow =
                    (const uint32_t *)(smem + s * STAGE_BYTES + A_BYTES + B_BYTES + r * lv_cols_of(NL)) + (o >> 2);
                uint32_t win[WW];
                uint32_t prev = lrow[0];
#pragma unroll
                for (int i = 0; i < WW; ++i) {
                    const uint32_t next = lrow[i + 1];
                    win[i] = __funnelshift_r(prev, next, 8 * (o & 3));
                    prev = next;
                }
                uint8_t *arow = smem + s * STAGE_BYTES + r * 128;
                const int n_valid = nb - t_kb;
                switch (v_kb) {
                case 0: onehot_kblock<NL, 0>(win, table, arow, r, n_valid); break;
                case 1: if constexpr (NL > 1) onehot_kblock<NL, 1>(win, table, arow, r, n_valid); break;
                case 2: if constexpr (NL > 2) onehot_kblock<NL, 2>(win, table, arow, r, n_valid); break;
                case 3: if constexpr (NL > 3) onehot_kblock<NL, 3>(win, table, arow, r, n_valid); break;
                default: if constexpr (NL > 4) onehot_kblock<NL, 4>(win, table, arow, r, n_valid); break;
                }
                // make the generic-proxy writes visible to the tensor core
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(full0 + 8 * s);
            }
        }
    }
    if (fail && g.err) atomicExch(g.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
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

// Tensor map of a row-major bf16 matrix [rows, ld] read in box_rows x 64 boxes.
int make_map(CUtensorMap *tm, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HESP_OK : HESP_ERR_ARG;
}

// Tensor map of int8 levels [rows, ld bytes] read in 128-row x box_cols-byte
// boxes (ld a multiple of 16; bytes past n_base read as 0).
int make_level_map(CUtensorMap *tm, const int8_t *ptr, int64_t rows, int64_t n_base, int64_t ld, int box_cols) {
    cuuint64_t dims[2] = {(cuuint64_t)n_base, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, BM};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<int8_t *>(ptr), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HESP_OK : HESP_ERR_ARG;
}

// Per-device launch state: the SM count and, per one-hot variant NL, whether
// the kernel's dynamic shared-memory limit has been raised on that device
// (a function attribute is per device).  Guarded by one mutex.
constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;
int g_sms[kMaxDevices] = {0};
bool g_attr_set[kMaxDevices][6] = {{false}};

template <int NL>
int prepare_device(int *sms) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HESP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (g_sms[dev] == 0 &&
        cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HESP_ERR_CUDA;
    if (!g_attr_set[dev][NL]) {
        if (cudaFuncSetAttribute(gemm_bf16_kernel<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_bytes_of(NL)) != cudaSuccess)
            return HESP_ERR_CUDA;
        g_attr_set[dev][NL] = true;
    }
    *sms = g_sms[dev];
    return HESP_OK;
}

template <int NL>
int launch_persistent(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap &tl, const GemmArgs &g,
                      cudaStream_t st) {
    constexpr int SMEM = smem_bytes_of(NL);
    int sms = 0;
    const int rc = prepare_device<NL>(&sms);
    if (rc) return rc;
    const int64_t tiles = (int64_t)((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
    const int64_t grid = tiles < sms ? tiles : sms;
    gemm_bf16_kernel<NL><<<(unsigned)grid, NL > 0 ? 320 + 128 * N_PROD_GROUPS : 320, SMEM, st>>>(ta, tb, tl, g);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
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
    if ((rc = make_map(&ta, A, g.M, g.K, lda, BM))) return rc;
    if ((rc = make_map(&tb, B, g.N, g.K, ldb, BN))) return rc;
    return launch_persistent<0>(ta, tb, tb, g, st);
}

// C = onehot(levels) . B^T with the one-hot A built in shared memory:
// A[r, f] = (levels[r * stride + f / NL] == f % NL) for f < n_base * NL, else 0;
// K = g.K (a multiple of 64, >= n_base * NL); levels 16-byte aligned with a
// row stride that is a multiple of 16 bytes (TMA reads the level windows).
int launch_gemm_onehot(const int8_t *levels, int64_t stride, int n_base, int NL, const void *B, int64_t ldb,
                       const GemmArgs &g0, cudaStream_t st) {
    if (g0.M < 1 || g0.N < 1 || g0.K < BK || g0.K % BK || (ldb & 7) || ldb < g0.K || !levels || NL < 1 ||
        NL > 5 || n_base < 1 || (int64_t)n_base * NL > g0.K || stride < n_base || (stride & 15))
        return HESP_ERR_ARG;
    if (((uintptr_t)B & 15) || ((uintptr_t)levels & 15)) return HESP_ERR_ARG;
    int rc = get_encode();
    if (rc) return rc;
    CUtensorMap tb, tl;
    if ((rc = make_map(&tb, B, g0.N, g0.K, ldb, BN))) return rc;
    if ((rc = make_level_map(&tl, levels, g0.M, n_base, stride, lv_cols_of(NL)))) return rc;
    GemmArgs g = g0;
    g.oh_lv = levels;
    g.oh_stride = stride;
    g.oh_base = n_base;
    g.oh_levels = NL;
    switch (NL) {
    case 1: return launch_persistent<1>(tb, tb, tl, g, st);
    case 2: return launch_persistent<2>(tb, tb, tl, g, st);
    case 3: return launch_persistent<3>(tb, tb, tl, g, st);
    case 4: return launch_persistent<4>(tb, tb, tl, g, st);
    default: return launch_persistent<5>(tb, tb, tl, g, st);
    }
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
