// Batched HeSP simulation kernel (sm_103a): one warp per candidate.
//
// For each candidate partition vector the warp
//   1. expands the tiled-Cholesky DAG (Sec. 1.1 Fig. 1 base loop, each base
//      task replaced by its 2x2 blocked algorithm `level` times, Sec. 2.1
//      "Recursive task partitioners") into packed task descriptors,
//   2. derives RaW/WaW/WaR dependences (Sec. 2.1) from per-atom last
//      writers and builds successor lists,
//   3. runs the event-driven FCFS + EFT-P schedule with write-back
//      (MSI-style) caching of accelerator memories and prefetching
//      transfers (Sec. 2.1 "Task and data scheduling heuristics"),
// and writes the makespan (int64 ns) and optionally the schedule.
//
// Lanes split the atoms of a task (data-ready times, transfer grouping,
// coherence updates), the processors (EFT evaluation; argmin by a packed
// (EFT << 6 | proc) key and two 32-bit warp reductions), the successors of a
// completed task and the words of the released-task bitmap.  A persistent
// grid pulls candidates from an atomic counter, so uneven candidates balance.
// Per-candidate state lives in a per-warp arena of the caller's workspace.
//
// Atoms are squares of side b >> Lc, Lc = the candidate's deepest split, so
// every data region of the DAG is a union of atoms, numbered in Z-order
// inside each upper-triangular tile: every region is one contiguous range.
//
// No thread ever waits on another warp; every loop is bounded (the event loop
// by an iteration cap that reports HESP_ERR_TIMEOUT).
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "hesp_internal.h"

namespace hesp {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kMaxL = HESP_MAX_LEVEL;
constexpr int kOpChol = 0, kOpTrsm = 1, kOpSyrk = 2, kOpGemm = 3;
constexpr int64_t kInf = INT64_MAX;

// Tasks produced by a task of each op split l times (2x2 blocked algorithms).
__constant__ int32_t c_cnt[4][kMaxL + 1] = {
    {1, 4, 20, 120, 816},    // chol: s(s+1)(s+2)/6, s = 2^l
    {1, 6, 40, 288, 2176},   // trsm: s^2(s+1)/2
    {1, 6, 40, 288, 2176},   // syrk: s^2(s+1)/2
    {1, 8, 64, 512, 4096}};  // gemm: s^3

// Children of a partitioned task in program order, and for each child region
// the (parent region, quadrant row, quadrant col) it is cut from, packed as
// region * 4 + row * 2 + col.  Regions: chol(A); trsm(T, B); syrk(A, C);
// gemm(A, B, C); the last region is the written one.
__constant__ int8_t c_nchild[4] = {4, 6, 6, 8};
__constant__ int8_t c_child_op[4][8] = {
    {kOpChol, kOpTrsm, kOpSyrk, kOpChol, 0, 0, 0, 0},
    {kOpTrsm, kOpTrsm, kOpGemm, kOpGemm, kOpTrsm, kOpTrsm, 0, 0},
    {kOpGemm, kOpSyrk, kOpSyrk, kOpGemm, kOpSyrk, kOpSyrk, 0, 0},
    {kOpGemm, kOpGemm, kOpGemm, kOpGemm, kOpGemm, kOpGemm, kOpGemm, kOpGemm}};
__constant__ int8_t c_child_sel[4][8][3] = {
    // chol(A): chol(A00); trsm(A00 -> A01); syrk(A01 -> A11); chol(A11)
    {{0, 0, 0}, {0, 1, 0}, {1, 3, 0}, {3, 0, 0}, {0}, {0}, {0}, {0}},
    // trsm(T, B): B := T^-T B
    {{0, 4, 0}, {0, 5, 0}, {1, 4, 6}, {1, 5, 7}, {3, 6, 0}, {3, 7, 0}, {0}, {0}},
    // syrk(A, C): C -= A^T A; k = 0, 1: gemm(Ak0, Ak1 -> C01); syrk(Ak0 -> C00); syrk(Ak1 -> C11)
    {{0, 1, 5}, {0, 4, 0}, {1, 7, 0}, {2, 3, 5}, {2, 4, 0}, {3, 7, 0}, {0}, {0}},
    // gemm(A, B, C): C -= A^T B; for k, i, j: gemm(Aki, Bkj -> Cij)
    {{0, 4, 8}, {0, 5, 9}, {1, 4, 10}, {1, 5, 11}, {2, 6, 8}, {2, 7, 9}, {3, 6, 10}, {3, 7, 11}}};

__device__ __forceinline__ int nreg_of(int op) { return op == kOpChol ? 1 : (op == kOpGemm ? 3 : 2); }

__device__ __forceinline__ uint32_t spread4(uint32_t v) {
    v = (v | (v << 2)) & 0x33u;
    v = (v | (v << 1)) & 0x55u;
    return v;
}

// Atom index of global atom coordinates (R, C) (R <= C tile-wise).
__device__ __forceinline__ uint32_t atom_index(int R, int C, int Lc, int n) {
    int I = R >> Lc, J = C >> Lc;
    uint32_t tile = (uint32_t)(I * n - (I * (I - 1)) / 2 + (J - I));
    uint32_t mask = (1u << Lc) - 1u;
    uint32_t z = (spread4((uint32_t)R & mask) << 1) | spread4((uint32_t)C & mask);
    return (tile << (2 * Lc)) | z;
}

// Decode base task t of the Fig. 1 loop on n tiles.
__device__ void decode_base(int n, int64_t t, int &op, int &K, int &I, int &J) {
    int k = 0;
    for (; k < n; ++k) {
        int64_t m = n - k - 1;
        int64_t S = 1 + 2 * m + (m * (m - 1)) / 2;
        if (t < S) break;
        t -= S;
    }
    int m = n - k - 1;
    K = k;
    if (t == 0) {
        op = kOpChol;
        I = J = k;
        return;
    }
    if (t <= m) {
        op = kOpTrsm;
        I = k;
        J = k + (int)t;
        return;
    }
    t -= m + 1;
    op = kOpSyrk;
    I = J = k;
    for (int i = k + 1; i < n; ++i) {
        int blk = n - i;
        if (t < blk) {
            if (t < blk - 1) {
                op = kOpGemm;
                I = i;
                J = i + 1 + (int)t;
            } else {
                op = kOpSyrk;
                I = J = i;
            }
            return;
        }
        t -= blk;
    }
}

// Descriptor of sub-task q of base task (op, K, I, J) split lvl times:
// op (2 bits) | lvl (3) | atom start of region 0, 1, 2 (19 bits each).
__device__ uint64_t decode_sub(int op, int K, int I, int J, int lvl, int q, int Lc, int n) {
    int R[3] = {0, 0, 0}, C[3] = {0, 0, 0};
    if (op == kOpChol) {
        R[0] = K; C[0] = K;
    } else if (op == kOpTrsm) {
        R[0] = K; C[0] = K; R[1] = K; C[1] = J;
    } else if (op == kOpSyrk) {
        R[0] = K; C[0] = I; R[1] = I; C[1] = I;
    } else {
        R[0] = K; C[0] = I; R[1] = K; C[1] = J; R[2] = I; C[2] = J;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        R[r] <<= Lc;
        C[r] <<= Lc;
    }
    int side = 1 << Lc;
    for (int d = lvl; d > 0; --d) {
        int nch = c_nchild[op];
        int ci = 0;
        for (; ci < nch - 1; ++ci) {
            int cc = c_cnt[c_child_op[op][ci]][d - 1];
            if (q < cc) break;
            q -= cc;
        }
        int cop = c_child_op[op][ci];
        int half = side >> 1;
        int nR[3] = {0, 0, 0}, nC[3] = {0, 0, 0};
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            int sel = c_child_sel[op][ci][r];
            int pr = sel >> 2, qp = (sel >> 1) & 1, qq = sel & 1;
            int baseR = pr == 0 ? R[0] : (pr == 1 ? R[1] : R[2]);
            int baseC = pr == 0 ? C[0] : (pr == 1 ? C[1] : C[2]);
            nR[r] = baseR + qp * half;
            nC[r] = baseC + qq * half;
        }
        op = cop;
        side = half;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R[r] = nR[r];
            C[r] = nC[r];
        }
    }
    int nr = nreg_of(op);
    uint64_t a0 = atom_index(R[0], C[0], Lc, n);
    uint64_t a1 = nr > 1 ? atom_index(R[1], C[1], Lc, n) : 0;
    uint64_t a2 = nr > 2 ? atom_index(R[2], C[2], Lc, n) : 0;
    return (uint64_t)op | ((uint64_t)lvl << 2) | (a0 << 5) | (a1 << 24) | (a2 << 43);
}

__device__ __forceinline__ uint32_t desc_atom(uint64_t d, int r) {
    return (uint32_t)((d >> (5 + 19 * r)) & 0x7FFFFu);
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Min over the warp of a non-negative 64-bit key, via two 32-bit reductions.
__device__ __forceinline__ uint64_t warp_min_u64(uint64_t k) {
    unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    unsigned hmin = __reduce_min_sync(FULL, hi);
    unsigned lmin = __reduce_min_sync(FULL, hi == hmin ? lo : 0xFFFFFFFFu);
    return ((uint64_t)hmin << 32) | lmin;
}

struct SimPtrs {
    uint64_t *desc;
    uint16_t *pending;
    int64_t *finish;
    int32_t *mark;  // aliases finish during dependence derivation
    int32_t *next;  // successor counts, then cursors, then per-processor FIFO links
    int32_t *succoff;
    int32_t *succ;
    int32_t *epred, *esucc;
    int32_t *lw;
    uint8_t *valid;
    int64_t *vfrom;
    uint32_t *bitmap;
    int64_t *xt;
};

struct KArgs {
    const hesp_cand *cands;
    const int8_t *levels;
    int64_t n_cand;
    int32_t max_tiles, max_level;
    int64_t *makespan;
    int32_t *status;
    int64_t *ntasks;
    const int64_t *sched_off;
    int16_t *sproc;
    int64_t *sstart, *sfinish;
    char *ws;
    Arena ar;
    int64_t n_slots;
};

template <int M>
struct AtomAcc {
    unsigned amax[M];   // latest (valid copy usable time - t) per memory, clamped to 0
    int cnt[M][M];      // atoms missing in m fetched from s
};

// Schedule task j at time t (EFT-P with data-ready times per memory).
// Returns false on an internal consistency failure.
template <int M, int NS>
__device__ __forceinline__ bool schedule_task(int j, int64_t t, const SimPtrs &P, int Lc, int lb_b, int lane,
                                               const int64_t *s_exec, const int8_t *s_pmem, const int8_t *s_ptype,
                                               int n_types, int pm[NS], int pt[NS], bool pv[NS], int64_t avail[NS],
                                               int head[NS], int tail[NS], int64_t hfin[NS], int64_t &mk,
                                               int16_t *sproc, int64_t *sstart, int64_t *sfinish) {
    const uint64_t d = P.desc[j];
    const int op = (int)(d & 3);
    const int lvl = (int)((d >> 2) & 7);
    const int nr = nreg_of(op);
    const int sh = 2 * (Lc - lvl);
    const int na = 1 << sh;
    const int tot = nr << sh;
    const int lb = lb_b - lvl;
    bool ok = true;

    int64_t drt_off[M];
    int64_t arr_off[M][M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        drt_off[m] = 0;
#pragma unroll
        for (int s = 0; s < M; ++s) arr_off[m][s] = 0;
    }
    if (M > 1) {
        AtomAcc<M> acc;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            acc.amax[m] = 0;
#pragma unroll
            for (int s = 0; s < M; ++s) acc.cnt[m][s] = 0;
        }
        for (int i0 = 0; i0 < tot; i0 += 32) {
            int i = i0 + lane;
            if (i < tot) {
                uint32_t x = desc_atom(d, i >> sh) + (uint32_t)(i & (na - 1));
                unsigned v = P.valid[x];
                int64_t vf[M];
#pragma unroll
                for (int m = 0; m < M; ++m) vf[m] = ((v >> m) & 1u) ? P.vfrom[(int64_t)x * M + m] : kInf;
                int src = -1;
#pragma unroll
                for (int s = M - 1; s >= 0; --s)
                    if (vf[s] <= t) src = s;
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    if ((v >> m) & 1u) {
                        int64_t dd = vf[m] - t;
                        if (dd > 0) {
                            if (dd > 0x7FFFFFFFLL) ok = false;
                            acc.amax[m] = max(acc.amax[m], (unsigned)min(dd, (int64_t)0x7FFFFFFF));
                        }
                    } else {
                        if (src < 0) ok = false;
#pragma unroll
                        for (int s = 0; s < M; ++s)
                            if (s == src) acc.cnt[m][s] += 1;
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            int64_t off = (int64_t)__reduce_max_sync(FULL, acc.amax[m]);
#pragma unroll
            for (int s = 0; s < M; ++s) {
                if (s == m) continue;
                int c = (int)__reduce_add_sync(FULL, (unsigned)acc.cnt[m][s]);
                if (c > 0) {
                    arr_off[m][s] = P.xt[c];
                    off = max(off, arr_off[m][s]);
                }
            }
            drt_off[m] = off;
        }
    }
    // EFT over processors; key = EFT << 6 | proc, ties to the lowest id.
    uint64_t key = ~0ull;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (pv[s]) {
            int64_t ex = s_exec[(op * HESP_MAX_TYPES + pt[s]) * HESP_LB + lb];
            int64_t ready = max(t, avail[s]);
            if (M > 1) {
                int64_t off = 0;
#pragma unroll
                for (int m = 0; m < M; ++m)
                    if (pm[s] == m) off = drt_off[m];
                ready = max(ready, t + off);
            }
            int64_t e = ready + ex;
            uint64_t k = ((uint64_t)e << 6) | (uint64_t)(lane + 32 * s);
            if (ex < 0 || e >= (1ll << 57)) ok = false;
            key = min(key, k);
        }
    }
    key = warp_min_u64(key);
    const int pbest = (int)(key & 63);
    const int64_t eft = (int64_t)(key >> 6);
    const int ms = s_pmem[pbest];
    const int64_t exb = s_exec[(op * HESP_MAX_TYPES + s_ptype[pbest]) * HESP_LB + lb];

    if (M > 1) {
        for (int i0 = 0; i0 < tot; i0 += 32) {
            int i = i0 + lane;
            if (i < tot) {
                int r = i >> sh;
                uint32_t x = desc_atom(d, r) + (uint32_t)(i & (na - 1));
                if (r == nr - 1) {
                    P.valid[x] = (uint8_t)(1u << ms);
                    P.vfrom[(int64_t)x * M + ms] = eft;
                } else {
                    unsigned v = P.valid[x];
                    if (!((v >> ms) & 1u)) {
                        int src = -1;
#pragma unroll
                        for (int s = M - 1; s >= 0; --s)
                            if (((v >> s) & 1u) && P.vfrom[(int64_t)x * M + s] <= t) src = s;
                        int64_t ao = 0;
#pragma unroll
                        for (int m = 0; m < M; ++m)
#pragma unroll
                            for (int s = 0; s < M; ++s)
                                if (m == ms && s == src) ao = arr_off[m][s];
                        P.valid[x] = (uint8_t)(v | (1u << ms));
                        P.vfrom[(int64_t)x * M + ms] = t + ao;
                    }
                }
            }
        }
    }
    if (lane == (pbest & 31)) {
        const int s = pbest >> 5;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            if (q == s) {
                avail[q] = eft;
                if (head[q] < 0) {
                    head[q] = j;
                    hfin[q] = eft;
                } else {
                    P.next[tail[q]] = j;
                }
                tail[q] = j;
            }
        }
    }
    if (lane == 0) {
        P.finish[j] = eft;
        P.next[j] = -1;
        if (sproc) {
            sproc[j] = (int16_t)pbest;
            sstart[j] = eft - exb;
            sfinish[j] = eft;
        }
    }
    mk = max(mk, eft);
    __syncwarp();
    return __all_sync(FULL, ok);
}

template <int M, int NS>
__global__ void __launch_bounds__(256) sim_kernel(DevPlatform pl, KArgs a, unsigned long long *work_counter) {
    __shared__ int64_t s_exec[4 * HESP_MAX_TYPES * HESP_LB];
    __shared__ int8_t s_pmem[HESP_MAX_PROCS];
    __shared__ int8_t s_ptype[HESP_MAX_PROCS];
    for (int i = threadIdx.x; i < 4 * HESP_MAX_TYPES * HESP_LB; i += blockDim.x) s_exec[i] = pl.exec[i];
    for (int i = threadIdx.x; i < HESP_MAX_PROCS; i += blockDim.x) {
        s_pmem[i] = pl.proc_mem[i];
        s_ptype[i] = pl.proc_type[i];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (slot >= a.n_slots) return;  // whole warp
    char *base = a.ws + slot * a.ar.slot_bytes;
    SimPtrs P;
    P.desc = (uint64_t *)(base + a.ar.off_desc);
    P.pending = (uint16_t *)(base + a.ar.off_pending);
    P.finish = (int64_t *)(base + a.ar.off_finish);
    P.mark = (int32_t *)(base + a.ar.off_finish);
    P.next = (int32_t *)(base + a.ar.off_next);
    P.succoff = (int32_t *)(base + a.ar.off_succoff);
    P.succ = (int32_t *)(base + a.ar.off_succ);
    P.epred = (int32_t *)(base + a.ar.off_epred);
    P.esucc = (int32_t *)(base + a.ar.off_esucc);
    P.lw = (int32_t *)(base + a.ar.off_lw);
    P.valid = (uint8_t *)(base + a.ar.off_valid);
    P.vfrom = (int64_t *)(base + a.ar.off_vfrom);
    P.bitmap = (uint32_t *)(base + a.ar.off_bitmap);
    P.xt = (int64_t *)(base + a.ar.off_xt);

    const int nprocs = pl.n_procs;
    int pm[NS], pt[NS];
    bool pv[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        int p = lane + 32 * s;
        pv[s] = p < nprocs;
        pm[s] = pv[s] ? pl.proc_mem[p] : 0;
        pt[s] = pv[s] ? pl.proc_type[p] : 0;
    }

    for (;;) {
        unsigned long long cl = 0;
        if (lane == 0) cl = atomicAdd(work_counter, 1ull);
        cl = __shfl_sync(FULL, cl, 0);
        if ((int64_t)cl >= a.n_cand) break;
        const int64_t c = (int64_t)cl;

        const hesp_cand cd = a.cands[c];
        const int n = cd.n_tiles;
        const int b = cd.b;
        const int64_t loff = cd.level_offset;
        int status = HESP_OK;
        int64_t T = 0;
        int64_t mk = 0;

        const bool bad_nb = n < 1 || n > a.max_tiles || b < 1 || (b & (b - 1)) != 0 || b > (1 << HESP_MAX_LOG2_BLOCK);
        const int64_t nb = bad_nb ? 0 : (int64_t)n * (n + 1) * (n + 2) / 6;
        int lmax = 0;
        bool badl = false;
        for (int64_t t0 = lane; t0 < nb; t0 += 32) {
            int l = a.levels[loff + t0];
            lmax = max(lmax, l);
            badl |= (l < 0 || l > a.max_level);
        }
        lmax = __reduce_max_sync(FULL, lmax);
        badl = __any_sync(FULL, badl);
        const int Lc = lmax;
        const int lb_b = bad_nb ? 0 : 31 - __clz(b);
        if (bad_nb || badl || (b >> Lc) < 1) status = HESP_ERR_ARG;

        const int64_t A = (int64_t)n * (n + 1) / 2 << (2 * Lc);
        if (status == HESP_OK && (A > a.ar.Acap || A >= (1 << 19))) status = HESP_ERR_CAPACITY;
        // task times used by this candidate must be representable
        if (status == HESP_OK) {
            bool bad = false;
            for (int e = lane; e < 4 * HESP_MAX_TYPES * (Lc + 1); e += 32) {
                int op = e / (HESP_MAX_TYPES * (Lc + 1));
                int rem = e % (HESP_MAX_TYPES * (Lc + 1));
                int ty = rem / (Lc + 1), l = rem % (Lc + 1);
                if (ty < pl.n_types && s_exec[(op * HESP_MAX_TYPES + ty) * HESP_LB + lb_b - l] < 0) bad = true;
            }
            if (__any_sync(FULL, bad)) status = HESP_ERR_ARG;
        }

        // ---- 1. count and expand tasks
        if (status == HESP_OK) {
            int64_t tcount = 0;
            for (int64_t t0 = 0; t0 < nb; t0 += 32) {
                int64_t t = t0 + lane;
                int cnt = 0;
                if (t < nb) {
                    int op, K, I, J;
                    decode_base(n, t, op, K, I, J);
                    cnt = c_cnt[op][a.levels[loff + t]];
                }
                tcount += __reduce_add_sync(FULL, (unsigned)cnt);
            }
            T = tcount;
            if (T > a.ar.Tcap || T >= INT_MAX / 2) status = HESP_ERR_CAPACITY;
        }
        if (status == HESP_OK) {
            int64_t off = 0;
            for (int64_t t0 = 0; t0 < nb; t0 += 32) {
                int64_t t = t0 + lane;
                int op = 0, K = 0, I = 0, J = 0, l = 0, cnt = 0;
                if (t < nb) {
                    decode_base(n, t, op, K, I, J);
                    l = a.levels[loff + t];
                    cnt = c_cnt[op][l];
                }
                const int incl = warp_incl_scan(cnt, lane);
                const int excl = incl - cnt;
                const int total = __shfl_sync(FULL, incl, 31);
                for (int g0 = 0; g0 < total; g0 += 32) {
                    const int g = g0 + lane;
                    // owner lane = first lane whose inclusive prefix exceeds g
                    int pos = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        int v = __shfl_sync(FULL, incl, pos + step - 1);
                        if (v <= g) pos += step;
                    }
                    const int owner = min(pos, 31);
                    const int q = g - __shfl_sync(FULL, excl, owner);
                    const int oop = __shfl_sync(FULL, op, owner);
                    const int oK = __shfl_sync(FULL, K, owner);
                    const int oI = __shfl_sync(FULL, I, owner);
                    const int oJ = __shfl_sync(FULL, J, owner);
                    const int ol = __shfl_sync(FULL, l, owner);
                    if (g < total) P.desc[off + g] = decode_sub(oop, oK, oI, oJ, ol, q, Lc, n);
                }
                off += total;
            }
            __syncwarp();
        }

        // ---- 2. dependences from per-atom last writers
        int64_t E = 0;
        if (status == HESP_OK) {
            for (int64_t x = lane; x < A; x += 32) P.lw[x] = -1;
            for (int64_t j = lane; j < T; j += 32) {
                P.mark[j] = -1;
                P.next[j] = 0;
            }
            __syncwarp();
            const unsigned lt_mask = (1u << lane) - 1u;
            for (int j = 0; j < (int)T; ++j) {
                const uint64_t d = P.desc[j];
                const int op = (int)(d & 3);
                const int lvl = (int)((d >> 2) & 7);
                const int nr = nreg_of(op);
                const int sh = 2 * (Lc - lvl);
                const int na = 1 << sh;
                const int tot = nr << sh;
                int cnt = 0;
                for (int i0 = 0; i0 < tot; i0 += 32) {
                    const int i = i0 + lane;
                    int w = -1;
                    if (i < tot) w = P.lw[desc_atom(d, i >> sh) + (uint32_t)(i & (na - 1))];
                    const unsigned grp = __match_any_sync(FULL, w);
                    bool isnew = false;
                    if (lane == __ffs(grp) - 1 && w >= 0 && P.mark[w] != j) {
                        P.mark[w] = j;
                        isnew = true;
                    }
                    const unsigned nm = __ballot_sync(FULL, isnew);
                    if (isnew) {
                        const int64_t e = E + cnt + __popc(nm & lt_mask);
                        if (e < a.ar.Ecap) {
                            P.epred[e] = w;
                            P.esucc[e] = j;
                        }
                        P.next[w] += 1;
                    }
                    cnt += __popc(nm);
                    __syncwarp();
                }
                if (lane == 0) P.pending[j] = (uint16_t)cnt;
                E += cnt;
                const uint32_t xw = desc_atom(d, nr - 1);
                for (int i = lane; i < na; i += 32) P.lw[xw + i] = j;
                __syncwarp();
            }
            if (E > a.ar.Ecap) status = HESP_ERR_CAPACITY;
        }

        // ---- 3. successor lists (CSR)
        if (status == HESP_OK) {
            int run = 0;
            for (int64_t j0 = 0; j0 < T; j0 += 32) {
                const int64_t j = j0 + lane;
                const int v = j < T ? P.next[j] : 0;
                const int incl = warp_incl_scan(v, lane);
                if (j < T) {
                    P.succoff[j] = run + incl - v;
                    P.next[j] = run + incl - v;
                }
                run += __shfl_sync(FULL, incl, 31);
            }
            if (lane == 0) P.succoff[T] = run;
            __syncwarp();
            for (int64_t e = lane; e < E; e += 32) {
                const int w = P.epred[e];
                const int pos = atomicAdd(&P.next[w], 1);
                P.succ[pos] = P.esucc[e];
            }
            __syncwarp();
        }

        // ---- 4. event-driven FCFS + EFT-P simulation
        if (status == HESP_OK) {
            if (M > 1) {
                for (int64_t x = lane; x < A; x += 32) {
                    P.valid[x] = 1;  // every atom valid in host memory from time 0
                    P.vfrom[x * M + 0] = 0;
                }
                // transfer time of k atoms (k * (b >> Lc)^2 elements)
                const int64_t ae = (int64_t)(b >> Lc) * (int64_t)(b >> Lc);
                const int kmax = 3 << (2 * Lc);
                for (int k = lane; k <= kmax; k += 32) {
                    const int64_t bytes = (int64_t)k * ae * pl.bpe;
                    P.xt[k] = k == 0 ? 0 : pl.lat + (bytes + pl.bw - 1) / pl.bw;
                }
            }
            const int W = (int)((T + 31) >> 5);
            int wlo = INT_MAX, whi = -1;
            for (int w0 = 0; w0 < W; w0 += 32) {
                // word w0 + q of the bitmap is built by a ballot over its 32 tasks
                for (int q = 0; q < 32 && w0 + q < W; ++q) {
                    const int64_t j = (int64_t)(w0 + q) * 32 + lane;
                    const bool rel = j < T && P.pending[j] == 0;
                    const unsigned bits = __ballot_sync(FULL, rel);
                    if (lane == 0) P.bitmap[w0 + q] = bits;
                    if (bits) {
                        wlo = min(wlo, w0 + q);
                        whi = max(whi, w0 + q);
                    }
                }
            }
            __syncwarp();

            int64_t avail[NS], hfin[NS];
            int head[NS], tail[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                avail[s] = 0;
                hfin[s] = kInf;
                head[s] = -1;
                tail[s] = -1;
            }
            int16_t *sproc = nullptr;
            int64_t *sstart = nullptr, *sfinish = nullptr;
            if (a.sched_off) {
                const int64_t so = a.sched_off[c];
                sproc = a.sproc + so;
                sstart = a.sstart + so;
                sfinish = a.sfinish + so;
            }
            int64_t t = 0;
            int64_t iters = 0;
            const int64_t iter_cap = 4 * T + 64;
            int64_t scheduled = 0;
            bool ok = true;
            for (;;) {
                // schedule every released task in ascending id
                for (int w0 = wlo; w0 <= whi && ok; w0 += 32) {
                    const int w = w0 + lane;
                    uint32_t bits = 0;
                    if (w <= whi) {
                        bits = P.bitmap[w];
                        if (bits) P.bitmap[w] = 0;
                    }
                    unsigned nz = __ballot_sync(FULL, bits != 0);
                    while (nz && ok) {
                        const int src = __ffs(nz) - 1;
                        nz &= nz - 1;
                        uint32_t wb = __shfl_sync(FULL, bits, src);
                        const int jb = (w0 + src) * 32;
                        while (wb && ok) {
                            const int bit = __ffs(wb) - 1;
                            wb &= wb - 1;
                            ok = schedule_task<M, NS>(jb + bit, t, P, Lc, lb_b, lane, s_exec, s_pmem, s_ptype,
                                                      pl.n_types, pm, pt, pv, avail, head, tail, hfin, mk, sproc,
                                                      sstart, sfinish);
                            ++scheduled;
                        }
                    }
                }
                if (!ok) {
                    status = HESP_ERR_STATE;
                    break;
                }
                wlo = INT_MAX;
                whi = -1;
                // next completion time
                uint64_t nk = ~0ull;
#pragma unroll
                for (int s = 0; s < NS; ++s) nk = min(nk, (uint64_t)hfin[s]);
                nk = warp_min_u64(nk);
                if (nk == (uint64_t)kInf) break;
                t = (int64_t)nk;
                if (++iters > iter_cap) {
                    status = HESP_ERR_TIMEOUT;
                    break;
                }
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    unsigned cm = __ballot_sync(FULL, hfin[s] == t);
                    while (cm) {
                        const int src = __ffs(cm) - 1;
                        cm &= cm - 1;
                        const int i = __shfl_sync(FULL, head[s], src);
                        const int e0 = P.succoff[i], e1 = P.succoff[i + 1];
                        int lo = INT_MAX, hi = -1;
                        for (int e = e0 + lane; e < e1; e += 32) {
                            const int sj = P.succ[e];
                            const int pvv = (int)P.pending[sj] - 1;
                            P.pending[sj] = (uint16_t)pvv;
                            if (pvv == 0) {
                                atomicOr(&P.bitmap[sj >> 5], 1u << (sj & 31));
                                lo = min(lo, sj >> 5);
                                hi = max(hi, sj >> 5);
                            }
                        }
                        wlo = min(wlo, __reduce_min_sync(FULL, lo));
                        whi = max(whi, __reduce_max_sync(FULL, hi));
                        if (lane == src) {
                            const int nx = P.next[i];
                            head[s] = nx;
                            hfin[s] = nx >= 0 ? P.finish[nx] : kInf;
                            if (nx < 0) tail[s] = -1;
                        }
                        __syncwarp();
                    }
                }
            }
            if (status == HESP_OK && scheduled != T) status = HESP_ERR_STATE;
        }

        if (lane == 0) {
            a.status[c] = status;
            a.makespan[c] = status == HESP_OK ? mk : -1;
            if (a.ntasks) a.ntasks[c] = T;
        }
    }
}

template <int M, int NS>
void occupancy_of(int *blocks) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, sim_kernel<M, NS>, 256, 0);
}

}  // namespace

int sim_kernel_occupancy(int n_mem, int n_procs, int *blocks_per_sm, int *threads_per_block) {
    *threads_per_block = 256;
    const bool two = n_procs > 32;
    switch (n_mem) {
    case 1: two ? occupancy_of<1, 2>(blocks_per_sm) : occupancy_of<1, 1>(blocks_per_sm); break;
    case 2: two ? occupancy_of<2, 2>(blocks_per_sm) : occupancy_of<2, 1>(blocks_per_sm); break;
    case 3: two ? occupancy_of<3, 2>(blocks_per_sm) : occupancy_of<3, 1>(blocks_per_sm); break;
    case 4: two ? occupancy_of<4, 2>(blocks_per_sm) : occupancy_of<4, 1>(blocks_per_sm); break;
    default: return HESP_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int launch_sim(const hesp_platform *p, const DevPlatform &dp, const Arena &ar, int64_t n_slots,
               const hesp_cand *cands, const int8_t *levels, int64_t n_cand, int32_t max_tiles, int32_t max_level,
               int64_t *makespan, int32_t *status, int64_t *ntasks, const int64_t *sched_off, int16_t *sproc,
               int64_t *sstart, int64_t *sfinish, char *ws, cudaStream_t stream) {
    KArgs a;
    a.cands = cands;
    a.levels = levels;
    a.n_cand = n_cand;
    a.max_tiles = max_tiles;
    a.max_level = max_level;
    a.makespan = makespan;
    a.status = status;
    a.ntasks = ntasks;
    a.sched_off = sched_off;
    a.sproc = sproc;
    a.sstart = sstart;
    a.sfinish = sfinish;
    a.ar = ar;
    a.n_slots = n_slots;
    a.ws = ws + kWsHeaderBytes;
    unsigned long long *ctr = &((WsHeader *)ws)->work_counter;
    if (cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), stream) != cudaSuccess) return HESP_ERR_CUDA;
    const int threads = 256;
    const int64_t blocks = (n_slots * 32 + threads - 1) / threads;
    const bool two = p->n_procs > 32;
    switch (p->n_mem) {
    case 1:
        if (two) sim_kernel<1, 2><<<(unsigned)blocks, threads, 0, stream>>>(dp, a, ctr);
        else sim_kernel<1, 1><<<(unsigned)blocks, threads, 0, stream>>>(dp, a, ctr);
        break;
    case 2:
        if (two) sim_kernel<2, 2><<<(unsigned)blocks, threads, 0, stream>>>(dp, a, ctr);
        else sim_kernel<2, 1><<<(unsigned)blocks, threads, 0, stream>>>(dp, a, ctr);
        break;
    case 3:
        if (two) sim_kernel<3, 2><<<(unsigned)blocks, threads, 0, stream>>>(dp, a, ctr);
        else sim_kernel<3, 1><<<(unsigned)blocks, threads, 0, stream>>>(dp, a, ctr);
        break;
    case 4:
        if (two) sim_kernel<4, 2><<<(unsigned)blocks, threads, 0, stream>>>(dp, a, ctr);
        else sim_kernel<4, 1><<<(unsigned)blocks, threads, 0, stream>>>(dp, a, ctr);
        break;
    default:
        return HESP_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

}  // namespace hesp
