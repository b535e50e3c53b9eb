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
#include <string.h>

#include <type_traits>

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

// The partition tables, copied to shared memory by every kernel that decodes
// tasks: lanes index them with different ops and levels, which the constant
// cache would serialise.
struct DecodeTables {
    int32_t cnt[4][kMaxL + 1];
    int8_t nchild[4];
    int8_t child_op[4][8];
    int8_t child_sel[4][8][3];
};

__device__ __forceinline__ void load_tables(DecodeTables &tb) {
    for (int i = threadIdx.x; i < 4 * (kMaxL + 1); i += blockDim.x)
        tb.cnt[i / (kMaxL + 1)][i % (kMaxL + 1)] = c_cnt[i / (kMaxL + 1)][i % (kMaxL + 1)];
    for (int i = threadIdx.x; i < 4; i += blockDim.x) tb.nchild[i] = c_nchild[i];
    for (int i = threadIdx.x; i < 32; i += blockDim.x) tb.child_op[i / 8][i % 8] = c_child_op[i / 8][i % 8];
    for (int i = threadIdx.x; i < 96; i += blockDim.x) tb.child_sel[i / 24][(i / 3) % 8][i % 3] = c_child_sel[i / 24][(i / 3) % 8][i % 3];
}

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

// Row-major position in the matrix (atom row * atoms per side + atom
// column) of dyadic atom x: the order finite memories break LRU ties in.
__device__ uint32_t rowmajor_of(uint32_t x, int Lc, int n) {
    const uint32_t tile = x >> (2 * Lc), z = x & ((1u << (2 * Lc)) - 1u);
    uint32_t r = 0, c = 0;
    for (int k = 0; k < Lc; ++k) {
        c |= ((z >> (2 * k)) & 1u) << k;
        r |= ((z >> (2 * k + 1)) & 1u) << k;
    }
    int I = 0;
    while (I + 1 < n && (uint32_t)((I + 1) * n - ((I + 1) * I) / 2) <= tile) ++I;
    const int J = (int)(tile - (uint32_t)(I * n - (I * (I - 1)) / 2)) + I;
    const uint32_t side = (uint32_t)n << Lc;
    return (((uint32_t)I << Lc) + r) * side + ((uint32_t)J << Lc) + c;
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
__device__ uint64_t decode_sub(int op, int K, int I, int J, int lvl, int q, int Lc, int n,
                               const DecodeTables &tb) {
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
        int nch = tb.nchild[op];
        int ci = 0;
        for (; ci < nch - 1; ++ci) {
            int cc = tb.cnt[tb.child_op[op][ci]][d - 1];
            if (q < cc) break;
            q -= cc;
        }
        int cop = tb.child_op[op][ci];
        int half = side >> 1;
        int nR[3] = {0, 0, 0}, nC[3] = {0, 0, 0};
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            int sel = tb.child_sel[op][ci][r];
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

// ---- one-level k-way partitions (Sec. 2.1: partition parameter p = 1 / k).
// A base task cut with factor k is replaced by its k-way blocked algorithm
// (chol: the Fig. 1 loop on k x k blocks; trsm, syrk, gemm: their block-row
// algorithms); mixed factors give non-dyadic tilings (Fig. 4).  Atoms are
// the common refinement of every tiling: a tile holds fL x fL atoms, fL the
// least common multiple of the candidate's factors, numbered row by row; a
// block of a k-way task is a w x w square of them, w = fL / k.

// Tasks of a base task of each op cut k ways.
__device__ __forceinline__ int fcount(int op, int k) {
    return op == kOpChol ? k * (k + 1) * (k + 2) / 6 : (op == kOpGemm ? k * k * k : k * k * (k + 1) / 2);
}

__device__ __forceinline__ uint32_t atom_index_f(int I, int J, int r, int c, int fL, int n) {
    const uint32_t tile = (uint32_t)(I * n - (I * (I - 1)) / 2 + (J - I));
    return tile * (uint32_t)(fL * fL) + (uint32_t)(r * fL + c);
}

// Descriptor of sub-task q of base task (op, K, I, J) cut k ways: op | k
// (in the level field) | first atom of each region.  Each region is block
// (br, bc) of one of the base task's tiles (tile index tr).
__device__ uint64_t decode_sub_f(int op, int K, int I, int J, int k, int q, int fL, int n) {
    int TR[3] = {0, 0, 0}, TC[3] = {0, 0, 0};
    if (op == kOpChol) {
        TR[0] = K; TC[0] = K;
    } else if (op == kOpTrsm) {
        TR[0] = K; TC[0] = K; TR[1] = K; TC[1] = J;
    } else if (op == kOpSyrk) {
        TR[0] = K; TC[0] = I; TR[1] = I; TC[1] = I;
    } else {
        TR[0] = K; TC[0] = I; TR[1] = K; TC[1] = J; TR[2] = I; TC[2] = J;
    }
    int sop = op;
    int tr[3] = {0, 1, 2}, br[3] = {0, 0, 0}, bc[3] = {0, 0, 0};
    int rem = q;
    if (k > 1 && op == kOpChol) {
        // for p: chol(App); for c > p: trsm(App -> Apc);
        //        for i > p: { for c > i: gemm(Api, Apc -> Aic); syrk(Api -> Aii) }
        tr[0] = tr[1] = tr[2] = 0;
        for (int p = 0; p < k; ++p) {
            if (rem == 0) { sop = kOpChol; br[0] = bc[0] = p; break; }
            rem -= 1;
            if (rem < k - 1 - p) { sop = kOpTrsm; br[0] = bc[0] = p; br[1] = p; bc[1] = p + 1 + rem; break; }
            rem -= k - 1 - p;
            bool done = false;
            for (int i = p + 1; i < k && !done; ++i) {
                const int ng = k - 1 - i;
                if (rem < ng) {
                    sop = kOpGemm;
                    br[0] = p; bc[0] = i; br[1] = p; bc[1] = i + 1 + rem; br[2] = i; bc[2] = i + 1 + rem;
                    done = true;
                } else if (rem == ng) {
                    sop = kOpSyrk;
                    br[0] = p; bc[0] = i; br[1] = i; bc[1] = i;
                    done = true;
                } else {
                    rem -= ng + 1;
                }
            }
            if (done) break;
        }
    } else if (k > 1 && op == kOpTrsm) {
        // for p: { for c: trsm(Tpp -> Bpc); for i > p: for c: gemm(Tpi, Bpc -> Bic) }
        for (int p = 0; p < k; ++p) {
            if (rem < k) { sop = kOpTrsm; br[0] = bc[0] = p; br[1] = p; bc[1] = rem; break; }
            rem -= k;
            const int ng = (k - 1 - p) * k;
            if (rem < ng) {
                const int i = p + 1 + rem / k, c = rem % k;
                sop = kOpGemm;
                tr[0] = 0; tr[1] = 1; tr[2] = 1;
                br[0] = p; bc[0] = i; br[1] = p; bc[1] = c; br[2] = i; bc[2] = c;
                break;
            }
            rem -= ng;
        }
    } else if (k > 1 && op == kOpSyrk) {
        // for p: for i: { for j > i: gemm(Api, Apj -> Cij); syrk(Api -> Cii) }
        bool done = false;
        for (int p = 0; p < k && !done; ++p)
            for (int i = 0; i < k && !done; ++i) {
                const int ng = k - 1 - i;
                if (rem < ng) {
                    sop = kOpGemm;
                    tr[0] = 0; tr[1] = 0; tr[2] = 1;
                    br[0] = p; bc[0] = i; br[1] = p; bc[1] = i + 1 + rem; br[2] = i; bc[2] = i + 1 + rem;
                    done = true;
                } else if (rem == ng) {
                    sop = kOpSyrk;
                    br[0] = p; bc[0] = i; br[1] = i; bc[1] = i;
                    done = true;
                } else {
                    rem -= ng + 1;
                }
            }
    } else if (k > 1) {
        // gemm: for p, i, j: gemm(Api, Bpj -> Cij)
        const int p = q / (k * k), i = (q / k) % k, j = q % k;
        br[0] = p; bc[0] = i; br[1] = p; bc[1] = j; br[2] = i; bc[2] = j;
    }
    const int w = fL / k;
    const int nr = nreg_of(sop);
    uint64_t at[3] = {0, 0, 0};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if (r < nr) {
            const int t = tr[r];
            const int tI = t == 0 ? TR[0] : (t == 1 ? TR[1] : TR[2]);
            const int tJ = t == 0 ? TC[0] : (t == 1 ? TC[1] : TC[2]);
            at[r] = atom_index_f(tI, tJ, br[r] * w, bc[r] * w, fL, n);
        }
    }
    return (uint64_t)sop | ((uint64_t)k << 2) | (at[0] << 5) | (at[1] << 24) | (at[2] << 43);
}

// Atom i (region-major) of a task's regions, and its region r.  Dyadic: a
// region is a contiguous run of 4^(Lc - lvl) = 1 << sh atoms (Z order);
// factor mode (fm): a w x w square of the tile's fL x fL atoms.
__device__ __forceinline__ uint32_t task_atom(uint64_t d, int i, int sh, int w, int fL, bool fm, int &r) {
    if (!fm) {
        r = i >> sh;
        return desc_atom(d, r) + (uint32_t)(i & ((1 << sh) - 1));
    }
    const int w2 = w * w;
    r = i / w2;
    const int q = i - r * w2;
    const int row = q / w;
    return desc_atom(d, r) + (uint32_t)(row * fL + (q - row * w));
}

// Index of a task's time in the exec tables: log2 of its block (dyadic), or
// its factor k (factor mode, tables laid out per k for the launch's b).
__device__ __forceinline__ int exec_idx(int lb_b, int lvl, bool fm) { return fm ? lvl : lb_b - lvl; }

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

// Max over the warp of a 64-bit unsigned value, via two 32-bit reductions.
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t k) {
    unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    unsigned hmax = __reduce_max_sync(FULL, hi);
    unsigned lmax = __reduce_max_sync(FULL, hi == hmax ? lo : 0u);
    return ((uint64_t)hmax << 32) | lmax;
}

// Per-processor FIFO of tasks in flight, threaded through the tasks: for a
// task in flight, its successor in the FIFO and that successor's finish time,
// read together (16 bytes) when it completes.  Record q also holds slot q of
// the FCFS wait queue of F-P / R-P (every task joins that queue once).
struct __align__(16) Link {
    int32_t next;
    int32_t rq;  // wait-queue slot
    int64_t nfin;
};
static_assert(sizeof(Link) == 16, "one 16-byte load per completion");

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
    int8_t *crit;  // optional: per base task, 1 if one of its tasks is on the critical path
    // 0: arenas per warp; 1 (keep): one arena per candidate, whose DAG is kept
    // for later launches; 2 (reuse): simulate the DAG a keep launch left there
    int32_t dag_mode;
    uint64_t layout_sig;  // identifies the arena layout of keep / reuse launches
    Arena ar;
    int64_t n_slots;
    int32_t bm_smem_words;  // > 0: the released-task bitmap lives in shared memory
    // 1: the levels array holds one partition factor k per base task (one-level
    // k-way partitions, every candidate of block size fm_b; max_level is the
    // largest factor); 0: dyadic split levels
    int32_t fmode, fm_b;
};

template <typename T>
__device__ __forceinline__ T *at(char *base, int64_t off) {
    return reinterpret_cast<T *>(base + off);
}

// Header of a candidate arena whose DAG is kept (keep / reuse launches).
struct KeptHeader {
    uint64_t sig;     // arena layout
    uint64_t lvhash;  // hash of the candidate (n, b, levels)
    int64_t T, E;     // tasks, dependence edges
    int32_t status;   // of the DAG build
    int32_t pad;
};

// Coherence state of one atom: for each memory the time from which its copy
// is usable there, or -1 if the memory holds no valid copy.  Stored as MP
// int64 per atom (MP = 2 for two memories, 4 for three or four).
template <int M>
struct AtomState {
    static constexpr int MP = M <= 2 ? 2 : 4;
    int64_t v[MP];
    __device__ __forceinline__ void load(const int64_t *p) {
        const longlong2 a = *reinterpret_cast<const longlong2 *>(p);
        v[0] = a.x;
        v[1] = a.y;
        if (MP == 4) {
            const longlong2 b = *reinterpret_cast<const longlong2 *>(p + 2);
            v[2] = b.x;
            v[3] = b.y;
        }
    }
    // lowest memory holding a copy usable at t, or -1
    __device__ __forceinline__ int source(int64_t t) const {
        int src = -1;
#pragma unroll
        for (int s = M - 1; s >= 0; --s)
            if (v[s] >= 0 && v[s] <= t) src = s;
        return src;
    }
    // memory whose copy is usable first (ties to the lowest), or -1
    __device__ __forceinline__ int earliest() const {
        int src = -1;
#pragma unroll
        for (int s = 0; s < M; ++s)
            if (v[s] >= 0 && (src < 0 || v[s] < v[src < 0 ? 0 : src])) src = s;
        return src;
    }
    // the source of a fetch at t: the lowest memory with a copy usable at t,
    // else (when copies may be in flight to their only holder: write-through,
    // write-around, write-backs of evictions) the copy usable first
    __device__ __forceinline__ int fetch_source(int64_t t, bool fallback) const {
        const int s = source(t);
        return (s < 0 && fallback) ? earliest() : s;
    }
};

// Packed per-(destination m, source s != m) atom counts: counter q =
// m * (M - 1) + (s < m ? s : s - 1), 10 bits each, three per word.
template <int M>
struct Counts {
    static constexpr int NQ = M * (M - 1);
    static constexpr int NW = (NQ + 2) / 3;  // three 10-bit counters per word (a task has <= 768 atoms)
    unsigned w[NW > 0 ? NW : 1];
    __device__ __forceinline__ static int q_of(int m, int s) { return m * (M - 1) + (s < m ? s : s - 1); }
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int k = 0; k < (NW > 0 ? NW : 1); ++k) w[k] = 0;
    }
    __device__ __forceinline__ void add(int m, int src) {
#pragma unroll
        for (int s = 0; s < M; ++s) {
            if (s == m) continue;
            const int q = q_of(m, s);
            if (s == src) w[q / 3] += 1u << (10 * (q % 3));
        }
    }
    __device__ __forceinline__ unsigned get(int m, int s) const {
        const int q = q_of(m, s);
        return (w[q / 3] >> (10 * (q % 3))) & 1023u;
    }
};

// Finite accelerator memories of one candidate (Sec. 2 "finite-size memory
// spaces"; the eviction rule is a reading, the paper gives none): bit m of
// `bounded` marks a finite memory that holds processors, cap[m] its
// capacity in atoms; use[x * MP + m] (arena) = the latest finish of a task
// that used atom x on a processor of memory m (-1: none).
struct CapState {
    unsigned bounded;
    int nA;  // atoms of the candidate
    int64_t cap[HESP_MAX_MEMS];
    int64_t occ[HESP_MAX_MEMS];  // atoms valid there now (kept exact at every commit)
};

// Schedule task j (descriptor d) at time t: data-ready time per memory, the processor
// choice `sel` (ties to the lowest id), commit of the coherence state (the
// caching policy `cache`), append to the chosen processor's FIFO.  Under
// F-P / R-P the caller guarantees a processor idle at t.  Clears `ok` on an
// internal inconsistency; sets `capfail` when no memory can take the task
// (finite memories, cs.bounded != 0: dyadic partitions, EFT-P / EIT-P).
template <int M, int NS, bool FIFO, bool REC, bool CAP>
__device__ __forceinline__ int64_t schedule_task(int j, uint64_t d, int64_t t, char *base, const KArgs &a, int Lc, int lb_b,
                                                 int fL, int lane, const int64_t *s_exec, const int8_t *s_pmem,
                                                 const int8_t *s_ptype, const int pm[NS], const int pt[NS],
                                                 const bool pv[NS], int64_t avail[NS], int head[NS], int tail[NS],
                                                 int64_t hfin[NS], int64_t &mk, bool &ok, int64_t sched_base,
                                                 int sel, uint64_t rp_seed, int cache, bool links, CapState &cs,
                                                 bool &capfail) {
    const int op = (int)(d & 3);
    const int lvl = (int)((d >> 2) & 7);
    const int nr = nreg_of(op);
    const bool fm = REC && fL > 0;          // factor mode: lvl is the factor k
    const int wf = fm ? fL / lvl : 0;       // block side in atoms (factor mode)
    const int sh = fm ? 0 : 2 * (Lc - lvl);
    const int na = fm ? wf * wf : 1 << sh;  // atoms per region
    const int tot = nr * na;
    const int lb = exec_idx(lb_b, lvl, fm);
    constexpr int MP = AtomState<M>::MP;
    int64_t *vfrom = at<int64_t>(base, a.ar.off_vfrom);
    // transfer time of k atoms: one table, or (links) one per ordered pair
    // of memories, table s * HESP_MAX_MEMS + d for messages s -> d
    const int64_t *xt = at<int64_t>(base, a.ar.off_xt);
    auto xtab = [&](int s, int d) -> const int64_t * {
        return links ? xt + (int64_t)(s * HESP_MAX_MEMS + d) * a.ar.Kcap : xt;
    };
    // finite memories in use; then, as under WT / WA, a copy may be valid
    // only in flight (a write-back), so a message departs when the last of
    // its data is usable at the source
    const bool capped = CAP && M > 1 && cs.bounded != 0;
    const bool fb = cache != HESP_CACHE_WB || capped;

    int64_t drt_off[M];
    Counts<M> cnt;
    cnt.clear();
#pragma unroll
    for (int m = 0; m < M; ++m) drt_off[m] = 0;
    // Leads over t (usable-from time - t).  Under FCFS a task starts once all
    // its predecessors finished, so a copy can lead t by one message time at
    // most (31 bits, else an error status); under the priority-list order a
    // copy issued for a task placed earlier may arrive far beyond t, so 64
    // bits.  dlead (write-through / write-around): lead of the departure of
    // the message m <- s, which leaves when the last of its data is usable at
    // the source.
    using Lead = typename std::conditional<FIFO, unsigned, uint64_t>::type;
    Lead dlead[M][M];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int s = 0; s < M; ++s) dlead[m][s] = 0;
    // finite memories: written atoms valid per memory before the commit
    unsigned wvalid[M];
#pragma unroll
    for (int m = 0; m < M; ++m) wvalid[m] = 0;
    if (M > 1) {
        // latest lead of a valid copy per memory
        Lead amax[M];
#pragma unroll
        for (int m = 0; m < M; ++m) amax[m] = 0;
        for (int i0 = 0; i0 < tot; i0 += 32) {
            const int i = i0 + lane;
            if (i < tot) {
                int rr;
                const uint32_t x = task_atom(d, i, sh, wf, fL, fm, rr);
                AtomState<M> st;
                st.load(vfrom + (int64_t)x * MP);
                if (capped && rr == nr - 1) {
#pragma unroll
                    for (int m = 1; m < M; ++m) wvalid[m] += st.v[m] >= 0;
                }
                const int src = st.fetch_source(t, fb);
                Lead slead = 0;  // lead of the source copy over t
                if (fb && src >= 0) {
#pragma unroll
                    for (int q = 0; q < M; ++q)
                        if (q == src && st.v[q] > t) {
                            const int64_t dl = st.v[q] - t;
                            if (FIFO) ok &= dl <= 0x7FFFFFFFLL;
                            slead = FIFO ? (Lead)min(dl, (int64_t)0x7FFFFFFF) : (Lead)dl;
                        }
                }
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    if (st.v[m] >= 0) {
                        const int64_t dd = st.v[m] - t;
                        if (dd > 0) {
                            if (FIFO) {
                                ok &= dd <= 0x7FFFFFFFLL;
                                amax[m] = max(amax[m], (Lead)min(dd, (int64_t)0x7FFFFFFF));
                            } else {
                                amax[m] = max(amax[m], (Lead)dd);
                            }
                        }
                    } else {
                        ok &= src >= 0;
                        cnt.add(m, src);
                        if (fb) {
#pragma unroll
                            for (int q = 0; q < M; ++q)
                                if (q == src) dlead[m][q] = max(dlead[m][q], slead);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < Counts<M>::NW; ++k) cnt.w[k] = __reduce_add_sync(FULL, cnt.w[k]);
        if (fb) {
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int q = 0; q < M; ++q)
                    if (q != m)
                        dlead[m][q] = FIFO ? (Lead)__reduce_max_sync(FULL, (unsigned)dlead[m][q])
                                           : (Lead)warp_max_u64((uint64_t)dlead[m][q]);
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            int64_t off = FIFO ? (int64_t)__reduce_max_sync(FULL, (unsigned)amax[m])
                               : (int64_t)warp_max_u64((uint64_t)amax[m]);
#pragma unroll
            for (int s = 0; s < M; ++s) {
                if (s == m) continue;
                const unsigned c = cnt.get(m, s);
                if (c > 0) off = max(off, (fb ? (int64_t)dlead[m][s] : 0) + xtab(s, m)[c]);
            }
            drt_off[m] = off;
        }
    }
    // Finite memories: memory m can take j when the atoms j lacks there fit
    // in its free space plus the atoms it may evict (valid there, not used by
    // j, no task in flight there still using them: use <= t).
    int64_t *const use = at<int64_t>(base, a.ar.off_use);
    unsigned feas = ~0u;  // bit m: memory m can take j
    int64_t need[M], room[M];
#pragma unroll
    for (int m = 0; m < M; ++m) need[m] = room[m] = 0;
    auto in_task = [&](uint32_t x) -> bool {
        bool in = false;
#pragma unroll
        for (int r = 0; r < 3; ++r)
            if (r < nr && x - desc_atom(d, r) < (uint32_t)na) in = true;
        return in;
    };
    if (capped) {
#pragma unroll
        for (int m = 1; m < M; ++m) {
            wvalid[m] = __reduce_add_sync(FULL, wvalid[m]);
            if (!((cs.bounded >> m) & 1u)) continue;
            unsigned nd = 0;
#pragma unroll
            for (int s = 0; s < M; ++s)
                if (s != m) nd += cnt.get(m, s);
            need[m] = nd;
            room[m] = cs.cap[m] - cs.occ[m];
            if (need[m] <= room[m]) continue;
            // count evictable atoms until there are enough
            const int64_t want = need[m] - room[m];
            int64_t got = 0;
            for (int x0 = 0; x0 < cs.nA && got < want; x0 += 32) {
                const int x = x0 + lane;
                const bool e = x < cs.nA && vfrom[(int64_t)x * MP + m] >= 0 &&
                               use[(int64_t)x * MP + m] <= t && !in_task((uint32_t)x);
                got += __popc(__ballot_sync(FULL, e));
            }
            if (got < want) feas &= ~(1u << m);
        }
    }
    // Processor choice, key = value << 6 | proc (ties to the lowest id):
    // EFT-P by the finish time, EIT-P by the time the processor is idle, F-P
    // by the task time among the processors idle at t, R-P 0 for the idle
    // processor whose rank in id order is the draw (1 for the others).
    int rp_pick = -1;
    unsigned ib[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) ib[s] = 0;
    if (sel >= HESP_SELECT_FP) {
        int n_idle = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            ib[s] = __ballot_sync(FULL, pv[s] && avail[s] <= t);
            n_idle += __popc(ib[s]);
        }
        if (sel == HESP_SELECT_RP && n_idle > 0)
            rp_pick = (int)lemire_draw(sm64_at(rp_seed, (uint64_t)j, 0), (uint32_t)n_idle);
    }
    uint64_t key = ~0ull;
    int64_t emine[NS];
    int before = 0;  // idle processors in lower slots
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        emine[s] = 0;
        const bool cand = pv[s] && (sel < HESP_SELECT_FP || avail[s] <= t) && ((feas >> pm[s]) & 1u);
        if (cand) {
            const int64_t ex = s_exec[(op * HESP_MAX_TYPES + pt[s]) * HESP_LB + lb];
            int64_t ready = max(t, avail[s]);
            const int64_t idle = ready;
            if (M > 1) {
                int64_t off = 0;
#pragma unroll
                for (int m = 0; m < M; ++m)
                    if (pm[s] == m) off = drt_off[m];
                ready = max(ready, t + off);
            }
            const int64_t e = ready + ex;
            emine[s] = e;
            ok &= ex >= 0 && e < (1ll << 57);
            int64_t v = e;
            if (sel == HESP_SELECT_EIT) v = idle;
            else if (sel == HESP_SELECT_FP) v = ex;
            else if (sel == HESP_SELECT_RP) v = (before + __popc(ib[s] & ((1u << lane) - 1u))) == rp_pick ? 0 : 1;
            key = min(key, ((uint64_t)v << 6) | (uint64_t)(lane + 32 * s));
        }
        if (sel >= HESP_SELECT_FP) before += __popc(ib[s]);
    }
    key = warp_min_u64(key);
    const bool none = sel >= HESP_SELECT_FP && key == ~0ull;  // no idle processor: the caller's error
    ok &= !none;
    if (capped && key == ~0ull) {  // no memory can take j
        capfail = true;
        key = 0;
    }
    const int pbest = none ? 0 : (int)(key & 63);
    int64_t eft = (int64_t)(key >> 6);
    if (sel != HESP_SELECT_EFT) {
        int64_t mine = emine[0];
#pragma unroll
        for (int s = 1; s < NS; ++s)
            if ((pbest >> 5) == s) mine = emine[s];
        eft = __shfl_sync(FULL, mine, pbest & 31);
    }
    const int ms = s_pmem[pbest];

    // Eviction from a finite memory: the least recently used evictable atom
    // (smallest use, ties to the lower atom) until j's missing atoms fit; an
    // evicted atom valid in no other memory goes back to host memory, all
    // in one message issued at t (marked -2 until its arrival is known).
    if (capped && !capfail && ((cs.bounded >> ms) & 1u) && need[ms] > room[ms]) {
        const int64_t k = need[ms] - room[ms];
        const int32_t *const rmk = at<int32_t>(base, a.ar.off_lw);
        for (int64_t q = 0; q < k; ++q) {
            // one pass: each lane's least (use, row-major key), then the warp's
            uint64_t bu = ~0ull;
            int bk = INT_MAX, bx = INT_MAX;
            for (int x = lane; x < cs.nA; x += 32) {
                if (vfrom[(int64_t)x * MP + ms] < 0) continue;
                const int64_t u = use[(int64_t)x * MP + ms];
                if (u > t || in_task((uint32_t)x)) continue;
                const int key = rmk[x];
                if ((uint64_t)u < bu || ((uint64_t)u == bu && key < bk)) {
                    bu = (uint64_t)u;
                    bk = key;
                    bx = x;
                }
            }
            const uint64_t best = warp_min_u64(bu);
            if (best == ~0ull) {
                ok = false;
                break;
            }
            const int vk = __reduce_min_sync(FULL, bu == best ? bk : INT_MAX);
            const int vx = __reduce_min_sync(FULL, (bu == best && bk == vk) ? bx : INT_MAX);
            if (lane == 0) {
                int64_t *pv2 = vfrom + (int64_t)vx * MP;
                bool elsewhere = false;
#pragma unroll
                for (int m = 0; m < M; ++m)
                    if (m != ms && pv2[m] >= 0) elsewhere = true;
                pv2[ms] = -1;
                if (!elsewhere) pv2[0] = -2;
            }
            __syncwarp();
        }
        cs.occ[ms] -= k;
        // write-backs: the atoms marked -2 in host memory
        unsigned nw = 0;
        for (int x = lane; x < cs.nA; x += 32) nw += vfrom[(int64_t)x * MP] == -2;
        const int n_wb = (int)__reduce_add_sync(FULL, nw);
        if (n_wb > 0) {
            const int64_t arrive = t + xtab(ms, 0)[n_wb];
            for (int x = lane; x < cs.nA; x += 32)
                if (vfrom[(int64_t)x * MP] == -2) vfrom[(int64_t)x * MP] = arrive;
        }
        __syncwarp();
    }

    if (M > 1) {
        for (int i0 = 0; i0 < tot; i0 += 32) {
            const int i = i0 + lane;
            if (i < tot) {
                int r;
                const uint32_t x = task_atom(d, i, sh, wf, fL, fm, r);
                int64_t *px = vfrom + (int64_t)x * MP;
                if (capped) {
                    int64_t *pu = use + (int64_t)x * MP + ms;
                    if (*pu < eft) *pu = eft;
                }
                if (r == nr - 1) {
                    // written block, every other copy invalidated: WB valid in
                    // the chosen memory from the finish; WT also in host memory
                    // from finish + xfer(block); WA (from an accelerator) only
                    // in host memory, from finish + xfer(block)
                    const bool acc = ms != 0 && cache != HESP_CACHE_WB;
                    const int64_t v_ms = (cache == HESP_CACHE_WA && ms != 0) ? -1 : eft;
                    const int64_t v_host = acc ? eft + xtab(ms, 0)[na] : -1;
                    longlong2 w0, w1;
                    w0.x = ms == 0 ? v_ms : v_host;
                    w0.y = ms == 1 ? v_ms : -1;
                    *reinterpret_cast<longlong2 *>(px) = w0;
                    if (MP == 4) {
                        w1.x = ms == 2 ? v_ms : -1;
                        w1.y = ms == 3 ? v_ms : -1;
                        *reinterpret_cast<longlong2 *>(px + 2) = w1;
                    }
                } else {
                    AtomState<M> st;
                    st.load(px);
                    int64_t vm = -1;
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        if (m == ms) vm = st.v[m];
                    if (vm < 0) {
                        // fetched: valid in the chosen memory from its message's arrival
                        const int src = st.fetch_source(t, fb);
                        unsigned c = 0;
                        int64_t lead = 0;
#pragma unroll
                        for (int m = 0; m < M; ++m)
#pragma unroll
                            for (int s = 0; s < M; ++s)
                                if (m != s && m == ms && s == src) {
                                    c = cnt.get(m, s);
                                    lead = (int64_t)dlead[m][s];
                                }
                        px[ms] = t + lead + xtab(src < 0 ? 0 : src, ms)[c];
                    }
                }
            }
        }
    }
    if (lane == (pbest & 31)) {
        Link *link = at<Link>(base, a.ar.off_link);
        const int s = pbest >> 5;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            if (q == s && !FIFO) avail[q] = eft;
            if (q == s && FIFO) {
                avail[q] = eft;
                if (head[q] < 0) {
                    head[q] = j;
                    hfin[q] = eft;
                } else {
                    link[tail[q]].next = j;
                    link[tail[q]].nfin = eft;
                }
                if (sel >= HESP_SELECT_FP) {
                    link[j].next = -1;  // record j's wait-queue slot stays
                } else {
                    // the whole record, so that reading it never needs DRAM
                    // for bytes that were never written
                    *reinterpret_cast<int4 *>(&link[j]) = make_int4(-1, 0, 0, 0);
                }
                tail[q] = j;
            }
        }
    }
    // REC: keep the chosen processor in the task's (spent) pending count for
    // the critical-path pass; a scheduled task's count is never read again
    if (REC && lane == 0) at<uint16_t>(base, a.ar.off_pending)[j] = (uint16_t)pbest;
    if (lane == 0 && sched_base >= 0) {
        a.sproc[sched_base + j] = (int16_t)pbest;
        a.sstart[sched_base + j] = eft - s_exec[(op * HESP_MAX_TYPES + s_ptype[pbest]) * HESP_LB + lb];
        a.sfinish[sched_base + j] = eft;
    }
    if (capped && !capfail) {
        // occupancy after the commit: j's missing atoms arrived in ms; its
        // written block left every other memory (and ms too under WA)
        if ((cs.bounded >> ms) & 1u) {
            cs.occ[ms] += need[ms];
            if (cache == HESP_CACHE_WA && ms != 0) cs.occ[ms] -= na;
        }
#pragma unroll
        for (int m = 1; m < M; ++m)
            if (m != ms && ((cs.bounded >> m) & 1u)) cs.occ[m] -= wvalid[m];
    }
    mk = max(mk, eft);
    __syncwarp();
    return eft;
}

// BUILD: expand and analyse each candidate's DAG and keep it (a keep launch
// without the simulation; platform independent, so one instantiation).
// CAP: the general instantiation with finite memories (kept apart so that
// the other general launches carry none of its registers).
// Registers: 64 per thread (8 four-warp CTAs per SM); with two processor
// slots per lane (more than 32 processors) 72, at 7 CTAs per SM (28 warps,
// still 4,144 resident candidates on 148 SMs), which removes nearly all of
// that instantiation's spills; the build launch 40 (six 8-warp CTAs).
template <int M, int NS, bool GEN, bool BUILD = false, bool CAP = false>
__global__ void __launch_bounds__(BUILD ? 256 : 128, BUILD ? 6 : (NS > 1 ? 7 : 8)) sim_kernel(DevPlatform pl, KArgs a,
                                                                 unsigned long long *work_counter) {
    __shared__ int64_t s_exec[4 * HESP_MAX_TYPES * HESP_LB];
    __shared__ int64_t s_wsum[4 * HESP_LB];
    __shared__ int8_t s_pmem[HESP_MAX_PROCS];
    __shared__ int8_t s_ptype[HESP_MAX_PROCS];
    __shared__ int s_info[8][32];  // dependence phase: per-lane atom info of the warp's round
    __shared__ DecodeTables s_tab;
    load_tables(s_tab);
    extern __shared__ uint32_t s_bitmap[];
    for (int i = threadIdx.x; i < 4 * HESP_MAX_TYPES * HESP_LB; i += blockDim.x) s_exec[i] = pl.exec[i];
    for (int i = threadIdx.x; i < 4 * HESP_LB; i += blockDim.x) s_wsum[i] = pl.wsum[i];
    for (int i = threadIdx.x; i < HESP_MAX_PROCS; i += blockDim.x) {
        s_pmem[i] = pl.proc_mem[i];
        s_ptype[i] = pl.proc_type[i];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const bool fm = GEN && a.fmode != 0;  // one-level k-way partitions
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (slot >= a.n_slots) return;  // whole warp
    char *const slot_base = a.ws + slot * a.ar.slot_bytes;
    constexpr int MP = AtomState<M>::MP;

    int pm[NS], pt[NS];
    bool pv[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int p = lane + 32 * s;
        pv[s] = p < pl.n_procs;
        pm[s] = pv[s] ? s_pmem[p] : 0;
        pt[s] = pv[s] ? s_ptype[p] : 0;
    }

    for (;;) {
        unsigned long long cl = 0;
        if (lane == 0) cl = atomicAdd(work_counter, 1ull);
        cl = __shfl_sync(FULL, cl, 0);
        if ((int64_t)cl >= a.n_cand) break;
        const int64_t c = (int64_t)cl;

        // keep / reuse launches address one arena per candidate
        char *const base = a.dag_mode ? a.ws + c * a.ar.slot_bytes : slot_base;
        uint32_t *const bm = a.bm_smem_words > 0 ? s_bitmap + (threadIdx.x >> 5) * a.bm_smem_words
                                                 : at<uint32_t>(base, a.ar.off_bitmap);
        const hesp_cand cd = a.cands[c];
        const int n = cd.n_tiles;
        const int b = cd.b;
        const int64_t loff = cd.level_offset;
        int status = HESP_OK;
        int64_t T = 0;
        int64_t mk = 0;

        const bool bad_nb = n < 1 || n > a.max_tiles || b < 1 || (!fm && (b & (b - 1)) != 0) ||
                            b > (1 << HESP_MAX_LOG2_BLOCK);
        const int64_t nb = bad_nb ? 0 : (int64_t)n * (n + 1) * (n + 2) / 6;
        int lmax = 0;
        unsigned fmask = 0;  // factor mode: the factors present
        bool badl = false;
        uint64_t lvh = 0;  // (keep / reuse) hash of the levels: sum of (l + 1) (t + 1) gamma
        for (int64_t t0 = lane; t0 < nb; t0 += 32) {
            const int l = a.levels[loff + t0];
            lmax = max(lmax, l);
            badl |= (l < (fm ? 1 : 0) || l > a.max_level);
            if (fm && l >= 1 && l <= 8) fmask |= 1u << l;
            lvh += (uint64_t)(l + 1) * ((uint64_t)(t0 + 1) * kGamma);
        }
        if (a.dag_mode) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) lvh += __shfl_xor_sync(FULL, lvh, o);
            lvh ^= ((uint64_t)(uint32_t)n << 32) ^ (uint64_t)(uint32_t)b;
        }
        lmax = __reduce_max_sync(FULL, lmax);
        badl = __any_sync(FULL, badl);
        // factor mode: a tile holds fL x fL atoms, fL = lcm of the factors
        int fL = 0;
        if (fm) {
            fmask = __reduce_or_sync(FULL, fmask);
            fL = 1;
            for (int f = 2; f <= 8; ++f)
                if ((fmask >> f) & 1u) {
                    int x = fL, y = f;
                    while (y) {
                        const int r = x % y;
                        x = y;
                        y = r;
                    }
                    fL = fL / x * f;
                }
        }
        const int Lc = fm ? 0 : lmax;
        const int lb_b = bad_nb ? 0 : 31 - __clz(b);
        if (bad_nb || badl || (b >> Lc) < 1) status = HESP_ERR_ARG;
        if (fm && status == HESP_OK && (b != a.fm_b || b % fL != 0)) status = HESP_ERR_ARG;

        const int64_t A = fm ? (int64_t)n * (n + 1) / 2 * fL * fL : (int64_t)n * (n + 1) / 2 << (2 * Lc);
        if (status == HESP_OK && (A > a.ar.Acap || A >= (1 << 19))) status = HESP_ERR_CAPACITY;
        // task times used by this candidate must be representable
        if (!BUILD && status == HESP_OK) {
            bool bad = false;
            const int nl = fm ? 9 : Lc + 1;  // levels 0..Lc, or factors 1..8
            for (int e = lane; e < 4 * HESP_MAX_TYPES * nl; e += 32) {
                const int op = e / (HESP_MAX_TYPES * nl);
                const int rem = e % (HESP_MAX_TYPES * nl);
                const int ty = rem / nl, l = rem % nl;
                const bool used = !fm || ((fmask >> l) & 1u) != 0;
                if (used && ty < pl.n_types && s_exec[(op * HESP_MAX_TYPES + ty) * HESP_LB + exec_idx(lb_b, l, fm)] < 0)
                    bad = true;
            }
            if (__any_sync(FULL, bad)) status = HESP_ERR_ARG;
        }

        // ---- 1. count and expand tasks
        const bool reuse = a.dag_mode == 2;
        uint64_t *const desc = at<uint64_t>(base, a.ar.off_desc);
        if (!reuse && status == HESP_OK) {
            int64_t tcount = 0;
            for (int64_t t0 = 0; t0 < nb; t0 += 32) {
                const int64_t t = t0 + lane;
                int cnt = 0;
                if (t < nb) {
                    int op, K, I, J;
                    decode_base(n, t, op, K, I, J);
                    const int l = a.levels[loff + t];
                    cnt = fm ? fcount(op, l) : s_tab.cnt[op][l];
                }
                tcount += __reduce_add_sync(FULL, (unsigned)cnt);
            }
            T = tcount;
            if (T > a.ar.Tcap || T >= INT_MAX / 2 || (a.bm_smem_words > 0 && ((T + 31) >> 5) > a.bm_smem_words))
                status = HESP_ERR_CAPACITY;
        }
        if (!reuse && status == HESP_OK) {
            int64_t off = 0;
            for (int64_t t0 = 0; t0 < nb; t0 += 32) {
                const int64_t t = t0 + lane;
                int op = 0, K = 0, I = 0, J = 0, l = 0, cnt = 0;
                if (t < nb) {
                    decode_base(n, t, op, K, I, J);
                    l = a.levels[loff + t];
                    cnt = fm ? fcount(op, l) : s_tab.cnt[op][l];
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
                        const int v = __shfl_sync(FULL, incl, pos + step - 1);
                        if (v <= g) pos += step;
                    }
                    const int owner = min(pos, 31);
                    const int q = g - __shfl_sync(FULL, excl, owner);
                    const int oop = __shfl_sync(FULL, op, owner);
                    const int oK = __shfl_sync(FULL, K, owner);
                    const int oI = __shfl_sync(FULL, I, owner);
                    const int oJ = __shfl_sync(FULL, J, owner);
                    const int ol = __shfl_sync(FULL, l, owner);
                    if (g < total)
                        desc[off + g] = fm ? decode_sub_f(oop, oK, oI, oJ, ol, q, fL, n)
                                           : decode_sub(oop, oK, oI, oJ, ol, q, Lc, n, s_tab);
                }
                off += total;
            }
            __syncwarp();
        }

        // ---- 2. dependences from per-atom last writers
        int64_t E = 0;
        if (!reuse && status == HESP_OK) {
            int32_t *const lw = at<int32_t>(base, a.ar.off_lw);
            int32_t *const mark = at<int32_t>(base, a.ar.off_succoff);  // offsets are built after this phase
            int32_t *const scnt = at<int32_t>(base, a.ar.off_next);
            // edges are appended grouped by successor, in creation order; only
            // the predecessor is stored (the successor is recovered from the
            // per-task counts when the successor lists are built)
            int32_t *const epred = at<int32_t>(base, a.ar.off_epred);
            uint16_t *const pending = at<uint16_t>(base, a.ar.off_pending);
            for (int64_t x = lane; x < A; x += 32) lw[x] = -1;
            for (int64_t j = lane; j < T; j += 32) {
                mark[j] = -1;
                scnt[j] = 0;
            }
            __syncwarp();
            const unsigned lt_mask = (1u << lane) - 1u;
            int *const info = s_info[threadIdx.x >> 5];  // per lane: (task in group << 1) | writes
            // Tasks are taken in creation order, as many consecutive ones per
            // round as have 32 atoms between them (one atom per lane).  The
            // last writer of an atom a task touches is the latest earlier
            // task of the round that writes it, else the last writer before
            // the round; a task whose atoms need more than one round is
            // taken alone (the per-task mark deduplicates across rounds).
            // (k-way partitions whose smallest tasks already fill a round are
            // taken one task at a time)
            const bool rounds = !fm || 3 * (fL / lmax) * (fL / lmax) <= 16;
            int j0 = 0;
            while (j0 < (int)T) {
                const int jt = j0 + lane;
                uint64_t dl = 0;
                int totl = 0;
                if (rounds && jt < (int)T) {
                    dl = desc[jt];
                    const int opl = (int)(dl & 3), lvll = (int)((dl >> 2) & 7);
                    const int wfl = fm ? fL / lvll : 0;
                    totl = nreg_of(opl) * (fm ? wfl * wfl : 1 << (2 * (Lc - lvll)));
                }
                const int incl = rounds ? warp_incl_scan(totl, lane) : 0;
                const int g = rounds ? __popc(__ballot_sync(FULL, jt < (int)T && incl <= 32)) : 0;  // tasks of the round
                if (g > 1) {
                    const int total = __shfl_sync(FULL, incl, g - 1);
                    // owner task of atom slot `lane`: first task lane whose inclusive count exceeds it
                    int pos = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int v = __shfl_sync(FULL, incl, pos + step - 1);
                        if (v <= lane) pos += step;
                    }
                    const int ob = min(pos, 31);
                    const bool act = lane < total;
                    const uint64_t d = __shfl_sync(FULL, dl, ob);
                    const int q = lane - (__shfl_sync(FULL, incl, ob) - __shfl_sync(FULL, totl, ob));
                    const int op = (int)(d & 3), lvl = (int)((d >> 2) & 7);
                    const int nr = nreg_of(op);
                    const int wf = fm ? fL / lvl : 0;
                    const int sh = fm ? 0 : 2 * (Lc - lvl);
                    int rr = 0;
                    const uint32_t x = act ? task_atom(d, q, sh, wf, fL, fm, rr) : 0u;
                    const bool wr = act && rr == nr - 1;
                    const int before = act ? lw[x] : -1;
                    info[lane] = (ob << 1) | (wr ? 1 : 0);
                    const unsigned peers = __match_any_sync(FULL, act ? (int)x : -1 - lane);
                    __syncwarp();
                    // latest writer of x among earlier tasks of the round, and the
                    // round's last writer of x (which updates the last-writer table)
                    int inw = -1, lastw = -1;
                    for (unsigned pm = peers; pm; pm &= pm - 1) {
                        const int v = info[__ffs(pm) - 1];
                        if (v & 1) {
                            const int pb = v >> 1;
                            if (pb < ob) inw = max(inw, pb);
                            lastw = max(lastw, pb);
                        }
                    }
                    const int pred = !act ? -1 : (inw >= 0 ? j0 + inw : before);
                    // one edge per distinct (task, predecessor)
                    const unsigned long long key = pred >= 0 ? ((unsigned long long)ob << 32) | (unsigned)pred
                                                             : ~0ull - (unsigned long long)lane;
                    const unsigned kg = __match_any_sync(FULL, key);
                    const bool emit = pred >= 0 && lane == __ffs(kg) - 1;
                    const unsigned em = __ballot_sync(FULL, emit);
                    if (emit) {
                        const int64_t e = E + __popc(em & lt_mask);
                        if (e < a.ar.Ecap) epred[e] = pred;
                        atomicAdd(&scnt[pred], 1);
                    }
                    E += __popc(em);
                    if (lane < g) {  // lane t: task j0 + t, its atom slots [incl - tot, incl)
                        const int lo = incl - totl;
                        const unsigned rm = (totl >= 32 ? ~0u : ((1u << totl) - 1u)) << lo;
                        pending[jt] = (uint16_t)__popc(em & rm);
                    }
                    __syncwarp();
                    if (wr && ob == lastw) lw[x] = j0 + ob;
                    __syncwarp();
                    j0 += g;
                    continue;
                }
                // task j0 alone (over several rounds when it has more than 32 atoms)
                const int j = j0;
                const uint64_t d = rounds ? __shfl_sync(FULL, dl, 0) : desc[j];
                const int op = (int)(d & 3);
                const int lvl = (int)((d >> 2) & 7);
                const int nr = nreg_of(op);
                const int wf = fm ? fL / lvl : 0;
                const int sh = fm ? 0 : 2 * (Lc - lvl);
                const int na = fm ? wf * wf : 1 << sh;
                const int tot = nr * na;
                const bool multi = tot > 32;  // one round: deduplicated inside the warp
                int cnt = 0;
                for (int i0 = 0; i0 < tot; i0 += 32) {
                    const int i = i0 + lane;
                    int w = -1;
                    int rr;
                    if (i < tot) w = lw[task_atom(d, i, sh, wf, fL, fm, rr)];
                    const unsigned grp = __match_any_sync(FULL, w);
                    bool isnew = lane == __ffs(grp) - 1 && w >= 0;
                    if (multi && isnew) {
                        if (mark[w] == j) isnew = false;
                        else mark[w] = j;
                    }
                    const unsigned nm = __ballot_sync(FULL, isnew);
                    if (isnew) {
                        const int64_t e = E + cnt + __popc(nm & lt_mask);
                        if (e < a.ar.Ecap) epred[e] = w;
                        atomicAdd(&scnt[w], 1);
                    }
                    cnt += __popc(nm);
                    __syncwarp();
                }
                if (lane == 0) pending[j] = (uint16_t)cnt;
                E += cnt;
                for (int i = lane; i < na; i += 32) {
                    int rr;
                    lw[task_atom(d, (nr - 1) * na + i, sh, wf, fL, fm, rr)] = j;
                }
                __syncwarp();
                j0 += 1;
            }
            if (E > a.ar.Ecap) status = HESP_ERR_CAPACITY;
        }

        // ---- 3. successor lists (CSR), each sorted by task id.  The sweep
        // appended pending[j] edges for task j, in creation order, so edge e
        // belongs to the successor whose prefix range of those counts holds e.
        if (!reuse && status == HESP_OK) {
            int32_t *const scnt = at<int32_t>(base, a.ar.off_next);
            int32_t *const succoff = at<int32_t>(base, a.ar.off_succoff);
            int32_t *const succ = at<int32_t>(base, a.ar.off_succ);
            const int32_t *const epred = at<int32_t>(base, a.ar.off_epred);
            const uint16_t *const npred = at<uint16_t>(base, a.ar.off_pending);
            int run = 0;
            for (int64_t j0 = 0; j0 < T; j0 += 32) {
                const int64_t j = j0 + lane;
                const int v = j < T ? scnt[j] : 0;
                const int incl = warp_incl_scan(v, lane);
                if (j < T) {
                    succoff[j] = run + incl - v;
                    scnt[j] = run + incl - v;
                }
                run += __shfl_sync(FULL, incl, 31);
            }
            if (lane == 0) succoff[T] = run;
            __syncwarp();
            int erun = 0;
            for (int64_t j0 = 0; j0 < T; j0 += 32) {
                const int64_t j = j0 + lane;
                const int k = j < T ? (int)npred[j] : 0;
                const int incl = warp_incl_scan(k, lane);
                const int total = __shfl_sync(FULL, incl, 31);
                for (int g0 = 0; g0 < total; g0 += 32) {
                    const int g = g0 + lane;
                    // successor lane = first lane whose inclusive count exceeds g
                    int pos = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int v = __shfl_sync(FULL, incl, pos + step - 1);
                        if (v <= g) pos += step;
                    }
                    // lanes of one predecessor take consecutive slots in lane
                    // (= successor) order, so every successor list is sorted by id
                    const int pr = g < total ? epred[erun + g] : -1 - lane;
                    const unsigned grp = __match_any_sync(FULL, pr);
                    const int lead = __ffs(grp) - 1;
                    int q0 = 0;
                    if (g < total && lane == lead) q0 = atomicAdd(&scnt[pr], __popc(grp));
                    q0 = __shfl_sync(FULL, q0, lead);
                    if (g < total) succ[q0 + __popc(grp & ((1u << lane) - 1u))] = (int)j0 + pos;
                    __syncwarp();
                }
                erun += total;
            }
            __syncwarp();
        }

        // ---- keep: save the DAG's state for reuse launches; reuse: check
        // that the kept DAG is this candidate's, then restore it
        if (a.dag_mode) {
            KeptHeader *const hd = at<KeptHeader>(base, a.ar.off_hdr);
            uint16_t *const pending = at<uint16_t>(base, a.ar.off_pending);
            uint16_t *const pend0 = at<uint16_t>(base, a.ar.off_pend0);
            if (!reuse) {
                if (status == HESP_OK)
                    for (int64_t j = lane; j < T; j += 32) pend0[j] = pending[j];
                if (lane == 0) {
                    hd->sig = a.layout_sig;
                    hd->lvhash = lvh;
                    hd->T = T;
                    hd->E = E;
                    hd->status = status;
                }
            } else if (status == HESP_OK) {
                const bool same = hd->sig == a.layout_sig && hd->lvhash == lvh && hd->T >= 0 && hd->T <= a.ar.Tcap &&
                                  hd->E >= 0 && hd->E <= a.ar.Ecap;
                if (!same) {
                    status = HESP_ERR_STATE;
                } else if (hd->status != HESP_OK) {
                    status = hd->status;
                } else {
                    T = hd->T;
                    E = hd->E;
                    for (int64_t j = lane; j < T; j += 32) pending[j] = pend0[j];
                }
            }
            __syncwarp();
        }

        // ---- 4. event-driven FCFS + EFT-P simulation
        if (!BUILD && status == HESP_OK) {
            uint16_t *const pending = at<uint16_t>(base, a.ar.off_pending);
            if (M > 1) {
                int64_t *const vfrom = at<int64_t>(base, a.ar.off_vfrom);
                for (int64_t x = lane; x < A; x += 32) {
                    // every atom valid in host memory from time 0, nowhere else
                    longlong2 v0;
                    v0.x = 0;
                    v0.y = -1;
                    *reinterpret_cast<longlong2 *>(vfrom + x * MP) = v0;
                    if (MP == 4) {
                        v0.x = -1;
                        *reinterpret_cast<longlong2 *>(vfrom + x * MP + 2) = v0;
                    }
                }
                // transfer time of k atoms (k * (b >> Lc)^2 elements): one
                // table, or (links) one per ordered pair of memories
                int64_t *const xt = at<int64_t>(base, a.ar.off_xt);
                const int64_t as = fm ? (int64_t)(b / fL) : (int64_t)(b >> Lc);
                const int64_t ae = as * as;
                const int kmax = fm ? 3 * fL * fL : 3 << (2 * Lc);
                for (int k = lane; k <= kmax; k += 32) {
                    const int64_t bytes = (int64_t)k * ae * pl.bpe;
                    xt[k] = k == 0 ? 0 : pl.lat + (bytes + pl.bw - 1) / pl.bw;
                }
                if (GEN && pl.use_links) {
                    for (int pr = 0; pr < M * M; ++pr) {
                        const int s = pr / M, d = pr % M;
                        if (s == d) continue;
                        int64_t *const xp = xt + (int64_t)(s * HESP_MAX_MEMS + d) * a.ar.Kcap;
                        const int64_t lat = pl.link_lat[s * HESP_MAX_MEMS + d];
                        const int64_t bw = pl.link_bw[s * HESP_MAX_MEMS + d];
                        for (int k = lane; k <= kmax; k += 32) {
                            const int64_t bytes = (int64_t)k * ae * pl.bpe;
                            xp[k] = k == 0 ? 0 : lat + (bytes + bw - 1) / bw;
                        }
                    }
                }
            }
            // finite accelerator memories (general instantiation, dyadic partitions)
            CapState cs;
            cs.bounded = 0;
            cs.nA = (int)A;
            bool capfail = false;
            if (CAP && M > 1 && pl.use_cap && !fm) {
                unsigned mm = 0;  // memories holding processors
#pragma unroll
                for (int s = 0; s < NS; ++s)
                    if (pv[s]) mm |= 1u << pm[s];
                mm = __reduce_or_sync(FULL, mm);
                const int64_t as = (int64_t)(b >> Lc);
                const int64_t abytes = as * as * pl.bpe;
#pragma unroll
                for (int m = 0; m < HESP_MAX_MEMS; ++m) {
                    cs.occ[m] = 0;  // every atom starts in host memory only
                    cs.cap[m] = m < M && pl.cap_bytes[m] > 0 ? pl.cap_bytes[m] / abytes : 0;
                    if (m > 0 && m < M && pl.cap_bytes[m] > 0 && ((mm >> m) & 1u)) cs.bounded |= 1u << m;
                }
                int64_t *const use = at<int64_t>(base, a.ar.off_use);
                for (int64_t x = lane; x < A * MP; x += 32) use[x] = -1;
                // LRU ties go to the lower row-major atom; the keys live in
                // the last-writer area, free after the dependence phase
                int32_t *const rmk = at<int32_t>(base, a.ar.off_lw);
                for (int64_t x = lane; x < A; x += 32) rmk[x] = (int32_t)rowmajor_of((uint32_t)x, Lc, n);
                __syncwarp();
            }
            // GEN = false: the FCFS + EFT-P + write-back instantiation; GEN =
            // true: every policy, chosen at run time from the platform.
            const int sel = GEN ? pl.select : HESP_SELECT_EFT;
            const bool waits = GEN && sel >= HESP_SELECT_FP;  // F-P, R-P: idle processors only
            const uint64_t rp_seed = pl.rp_seed;
            const int cache = GEN ? pl.cache : HESP_CACHE_WB;
            const bool links = GEN && pl.use_links;
            if (GEN && pl.order == HESP_ORDER_PL) {
                // ---- PL: a priority list by critical time (HEFT-like); each task
                // is scheduled at its release time, the latest finish among its
                // predecessors.  Critical times, release times and the two sort
                // buffers use the FIFO link area (no FIFOs in this order).
                int64_t *const crit = at<int64_t>(base, a.ar.off_link);
                int64_t *const rel = crit + T;
                uint64_t *const keyA = reinterpret_cast<uint64_t *>(crit + 2 * T);
                uint64_t *const keyB = reinterpret_cast<uint64_t *>(crit + 3 * T);
                uint32_t *const hist = at<uint32_t>(base, a.ar.off_hist);
                const int32_t *const succoff = at<int32_t>(base, a.ar.off_succoff);
                const int32_t *const succ = at<int32_t>(base, a.ar.off_succ);
                const unsigned lt_mask = (1u << lane) - 1u;
                bool okp = T < (1 << 22);
                // critical time = time summed over the processors + largest successor's, backwards
                for (int j = (int)T - 1; j >= 0 && okp; --j) {
                    const uint64_t d = desc[j];
                    const int e0 = succoff[j], e1 = succoff[j + 1];
                    uint64_t mx = 0;
                    for (int e = e0 + lane; e < e1; e += 32) mx = max(mx, (uint64_t)crit[succ[e]]);
                    mx = warp_max_u64(mx);
                    const int64_t w = s_wsum[(int)(d & 3) * HESP_LB + exec_idx(lb_b, (int)((d >> 2) & 7), fm)];
                    const int64_t cj = (int64_t)mx + w;
                    okp = okp && w > 0 && cj < (1ll << 41);
                    if (lane == 0) crit[j] = cj;
                    __syncwarp();
                }
                // sort keys (2^41 - 1 - crit) << 22 | id ascending: decreasing critical time, then id
                for (int64_t j = lane; j < T && okp; j += 32) {
                    keyA[j] = ((uint64_t)((1ll << 41) - 1 - crit[j]) << 22) | (uint64_t)j;
                    rel[j] = 0;
                }
                __syncwarp();
                uint64_t *src = keyA, *dst = keyB;
                for (int pass = 0; pass < 8 && okp; ++pass) {  // LSD radix sort, 8-bit digits
                    const int sh = pass * 8;
                    for (int k = lane; k < 256; k += 32) hist[k] = 0;
                    __syncwarp();
                    for (int64_t i = lane; i < T; i += 32) atomicAdd(&hist[(src[i] >> sh) & 255], 1u);
                    __syncwarp();
                    uint32_t v[8], sum = 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        v[q] = hist[lane * 8 + q];
                        sum += v[q];
                    }
                    uint32_t run = (uint32_t)warp_incl_scan((int)sum, lane) - sum;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        hist[lane * 8 + q] = run;
                        run += v[q];
                    }
                    __syncwarp();
                    for (int64_t i0 = 0; i0 < T; i0 += 32) {
                        const int64_t i = i0 + lane;
                        const bool act = i < T;
                        const uint64_t k = act ? src[i] : 0;
                        const int dg = act ? (int)((k >> sh) & 255) : 256 + lane;
                        const unsigned grp = __match_any_sync(FULL, dg);
                        const int rank = __popc(grp & lt_mask);
                        const uint32_t b0 = act ? hist[dg] : 0;
                        __syncwarp();
                        if (act) {
                            dst[b0 + rank] = k;
                            if (rank == 0) hist[dg] = b0 + __popc(grp);
                        }
                        __syncwarp();
                    }
                    uint64_t *tmp = src;
                    src = dst;
                    dst = tmp;
                }
                int64_t avail[NS], hfin[NS];
                int head[NS], tail[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    avail[s] = 0;
                    hfin[s] = kInf;
                    head[s] = -1;
                    tail[s] = -1;
                }
                const int64_t sched_base = a.sched_off ? a.sched_off[c] : -1;
                bool ok = true;
                for (int64_t q = 0; q < T && okp; ++q) {
                    const int j = (int)(src[q] & ((1u << 22) - 1));
                    int64_t tj = rel[j];
                    if (waits) {
                        // no processor idle at the release time: the first one to become idle
                        bool any = false;
                        uint64_t mn = ~0ull;
#pragma unroll
                        for (int s = 0; s < NS; ++s)
                            if (pv[s]) {
                                any |= avail[s] <= tj;
                                mn = min(mn, (uint64_t)avail[s]);
                            }
                        if (!__any_sync(FULL, any)) tj = (int64_t)warp_min_u64(mn);
                    }
                    const int64_t fj = schedule_task<M, NS, false, GEN, CAP>(j, desc[j], tj, base, a, Lc, lb_b, fL, lane, s_exec, s_pmem,
                                                                   s_ptype, pm, pt, pv, avail, head, tail, hfin, mk,
                                                                   ok, sched_base, sel, rp_seed, cache, links, cs, capfail);
                    const int e0 = succoff[j], e1 = succoff[j + 1];
                    for (int e = e0 + lane; e < e1; e += 32) {
                        const int sj = succ[e];
                        if (fj > rel[sj]) rel[sj] = fj;
                    }
                    __syncwarp();
                }
                if (!__all_sync(FULL, ok && okp)) status = HESP_ERR_STATE;
                if (capfail) status = HESP_ERR_CAPACITY;
            } else {
            const int W = (int)((T + 31) >> 5);
            int wlo = INT_MAX, whi = -1;
            for (int w0 = 0; w0 < W; w0 += 32) {
                // word w0 + q of the bitmap is built by a ballot over its 32 tasks
                for (int q = 0; q < 32 && w0 + q < W; ++q) {
                    const int64_t j = (int64_t)(w0 + q) * 32 + lane;
                    const bool rel = j < T && pending[j] == 0;
                    const unsigned bits = __ballot_sync(FULL, rel);
                    if (lane == 0) bm[w0 + q] = bits;
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
            const int64_t sched_base = a.sched_off ? a.sched_off[c] : -1;
            const int32_t *const succoff = at<int32_t>(base, a.ar.off_succoff);
            const int32_t *const succ = at<int32_t>(base, a.ar.off_succ);
            Link *const link = at<Link>(base, a.ar.off_link);
            int qh = 0, qt = 0;  // F-P / R-P wait queue: link[qh .. qt).rq
            int64_t t = 0;
            int iters = 0;
            const int iter_cap = 4 * (int)T + 64;
            int scheduled = 0;
            bool ok = true;
            // Tasks released when a single task completes are taken straight
            // from its (sorted) successor list; those released by several
            // completions at one time wait in the bitmap.
            for (;;) {
                // schedule every task the bitmap holds, in ascending id
                {
                    for (int w0 = wlo; w0 <= whi; w0 += 32) {
                        const int w = w0 + lane;
                        uint32_t bits = 0;
                        if (w <= whi) {
                            bits = bm[w];
                            if (bits) bm[w] = 0;
                        }
                        unsigned nz = __ballot_sync(FULL, bits != 0);
                        while (nz) {
                            const int src = __ffs(nz) - 1;
                            nz &= nz - 1;
                            uint32_t wb = __shfl_sync(FULL, bits, src);
                            const int jb = (w0 + src) * 32;
                            // the descriptors of the word's released tasks, one per lane, in one round trip
                            const uint64_t dw = ((wb >> lane) & 1u) ? desc[jb + lane] : 0ull;
                            while (wb) {
                                const int bit = __ffs(wb) - 1;
                                wb &= wb - 1;
                                if (waits) {
                                    if (lane == 0) link[qt].rq = jb + bit;
                                    ++qt;
                                    continue;
                                }
                                schedule_task<M, NS, true, GEN, CAP>(jb + bit, __shfl_sync(FULL, dw, bit), t, base, a, Lc, lb_b, fL, lane, s_exec, s_pmem, s_ptype,
                                                           pm, pt, pv, avail, head, tail, hfin, mk, ok, sched_base,
                                                           sel, rp_seed, cache, links, cs, capfail);
                                ++scheduled;
                            }
                        }
                    }
                    wlo = INT_MAX;
                    whi = -1;
                }
                if (waits) {
                    // serve the queue from its front while some processor is idle at t
                    __syncwarp();
                    while (qh < qt) {
                        bool any = false;
#pragma unroll
                        for (int s = 0; s < NS; ++s) any |= pv[s] && avail[s] <= t;
                        if (!__any_sync(FULL, any)) break;
                        const int j = link[qh].rq;
                        ++qh;
                        schedule_task<M, NS, true, GEN, CAP>(j, desc[j], t, base, a, Lc, lb_b, fL, lane, s_exec, s_pmem, s_ptype, pm, pt, pv,
                                                   avail, head, tail, hfin, mk, ok, sched_base, sel, rp_seed, cache, links, cs, capfail);
                        ++scheduled;
                    }
                }
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
                unsigned cms[NS];
                int ncomp = 0;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    cms[s] = __ballot_sync(FULL, hfin[s] == t);
                    ncomp += __popc(cms[s]);
                }
                if (ncomp == 1) {
                    // the only completion: its processor's FIFO advances, then
                    // its successors, 32 at a time in ascending id, lose one
                    // pending predecessor, and the released ones are scheduled
                    // (F-P / R-P: queued) in lane order
                    int src = 0, i = 0;
#pragma unroll
                    for (int s = 0; s < NS; ++s)
                        if (cms[s]) {
                            src = __ffs(cms[s]) - 1;
                            i = __shfl_sync(FULL, head[s], src);
                        }
                    Link l0;
                    l0.next = 0;
                    l0.nfin = 0;
                    if (lane == src) l0 = link[i];
                    const int eq = lane < 2 ? succoff[i + lane] : 0;
                    const int e0 = __shfl_sync(FULL, eq, 0), e1 = __shfl_sync(FULL, eq, 1);
                    if (lane == src) {
#pragma unroll
                        for (int s = 0; s < NS; ++s)
                            if (cms[s]) {
                                head[s] = l0.next;
                                hfin[s] = l0.next >= 0 ? l0.nfin : kInf;
                                if (l0.next < 0) tail[s] = -1;
                            }
                    }
                    __syncwarp();
                    for (int c0 = e0; c0 < e1; c0 += 32) {
                        const int e = c0 + lane;
                        int sj = 0;
                        uint64_t dsj = 0;
                        bool relj = false;
                        if (e < e1) {
                            sj = succ[e];
                            // the descriptor is read beside the count (one
                            // round trip instead of two for a released task)
                            dsj = desc[sj];
                            const int pvv = (int)pending[sj] - 1;
                            pending[sj] = (uint16_t)pvv;
                            relj = pvv == 0;
                        }
                        unsigned rel = __ballot_sync(FULL, relj);
                        while (rel) {
                            const int bl = __ffs(rel) - 1;
                            rel &= rel - 1;
                            const int j = __shfl_sync(FULL, sj, bl);
                            const uint64_t dj = __shfl_sync(FULL, dsj, bl);
                            if (waits) {
                                if (lane == 0) link[qt].rq = j;
                                ++qt;
                                continue;
                            }
                            schedule_task<M, NS, true, GEN, CAP>(j, dj, t, base, a, Lc, lb_b, fL, lane, s_exec, s_pmem,
                                                               s_ptype, pm, pt, pv, avail, head, tail, hfin, mk, ok,
                                                               sched_base, sel, rp_seed, cache, links, cs, capfail);
                            ++scheduled;
                        }
                    }
                    __syncwarp();
                    continue;
                }
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    unsigned cm = cms[s];
                    while (cm) {
                        const int src = __ffs(cm) - 1;
                        cm &= cm - 1;
                        const int i = __shfl_sync(FULL, head[s], src);
                        // lane src: the FIFO record; lanes 0, 1: the successor range
                        Link l0;
                        l0.next = 0;
                        l0.nfin = 0;
                        if (lane == src) l0 = link[i];
                        const int eq = lane < 2 ? succoff[i + lane] : 0;
                        const int e0 = __shfl_sync(FULL, eq, 0), e1 = __shfl_sync(FULL, eq, 1);
                        {
                            int lo = INT_MAX, hi = -1;
                            for (int e = e0 + lane; e < e1; e += 32) {
                                const int sj = succ[e];
                                const int pvv = (int)pending[sj] - 1;
                                pending[sj] = (uint16_t)pvv;
                                if (pvv == 0) {
                                    atomicOr(&bm[sj >> 5], 1u << (sj & 31));
                                    lo = min(lo, sj >> 5);
                                    hi = max(hi, sj >> 5);
                                }
                            }
                            wlo = min(wlo, __reduce_min_sync(FULL, lo));
                            whi = max(whi, __reduce_max_sync(FULL, hi));
                        }
                        if (lane == src) {
                            head[s] = l0.next;
                            hfin[s] = l0.next >= 0 ? l0.nfin : kInf;
                            if (l0.next < 0) tail[s] = -1;
                        }
                        __syncwarp();
                    }
                }
            }
            if (!__all_sync(FULL, ok)) status = HESP_ERR_STATE;
            if (status == HESP_OK && scheduled != T) status = HESP_ERR_STATE;
            if (capfail) status = HESP_ERR_CAPACITY;
            }
        }

        // ---- 5. critical-path flags per base task: a task is critical when the
        // longest path through it, weighted by the scheduled task times, is as
        // long as the longest path of the DAG (the iterative solver's CP choice)
        if (!BUILD && GEN && a.crit && status == HESP_OK) {
            const uint16_t *const prc = at<uint16_t>(base, a.ar.off_pending);
            const int32_t *const succoff = at<int32_t>(base, a.ar.off_succoff);
            const int32_t *const succ = at<int32_t>(base, a.ar.off_succ);
            int64_t *const down = at<int64_t>(base, a.ar.off_link);  // the link area is free now
            int64_t *const up = down + T;
            auto dur = [&](int64_t j) -> int64_t {
                const uint64_t d = desc[j];
                return s_exec[((int)(d & 3) * HESP_MAX_TYPES + s_ptype[prc[j]]) * HESP_LB +
                              exec_idx(lb_b, (int)((d >> 2) & 7), fm)];
            };
            // longest path from each task to a sink (creation order is topological)
            for (int64_t j = T - 1; j >= 0; --j) {
                uint64_t mx = 0;
                for (int e = succoff[j] + lane; e < succoff[j + 1]; e += 32) mx = max(mx, (uint64_t)down[succ[e]]);
                mx = warp_max_u64(mx);
                if (lane == 0) down[j] = dur(j) + (int64_t)mx;
                __syncwarp();
            }
            // longest path from a source to each task, pushed along the successor lists
            for (int64_t j = lane; j < T; j += 32) up[j] = dur(j);
            __syncwarp();
            uint64_t lmax = 0;
            for (int64_t j = 0; j < T; ++j) {
                const int64_t uj = up[j];
                for (int e = succoff[j] + lane; e < succoff[j + 1]; e += 32) {
                    const int s = succ[e];
                    up[s] = max(up[s], uj + dur(s));
                }
                __syncwarp();
            }
            for (int64_t j = lane; j < T; j += 32) lmax = max(lmax, (uint64_t)down[j]);
            const int64_t longest = (int64_t)warp_max_u64(lmax);
            // base tasks own consecutive task ranges in creation order
            int64_t run = 0;
            for (int64_t t0 = 0; t0 < nb; t0 += 32) {
                const int64_t t = t0 + lane;
                int cnt = 0;
                if (t < nb) {
                    int op, K, I, J;
                    decode_base(n, t, op, K, I, J);
                    const int l = a.levels[loff + t];
                    cnt = fm ? fcount(op, l) : s_tab.cnt[op][l];
                }
                const int incl = warp_incl_scan(cnt, lane);
                if (t < nb) {
                    int8_t f = 0;
                    for (int64_t j = run + incl - cnt; j < run + incl && !f; ++j)
                        f = (up[j] + down[j] - dur(j) == longest) ? 1 : 0;
                    a.crit[loff + t] = f;
                }
                run += __shfl_sync(FULL, incl, 31);
            }
            __syncwarp();
        }

        if (lane == 0) {
            a.status[c] = status;
            if (a.makespan) a.makespan[c] = status == HESP_OK ? mk : -1;
            if (a.ntasks) a.ntasks[c] = T;
        }
        __syncwarp();
    }
}

// Simulation launches use CTAs of four candidate warps: a batch smaller than
// the resident capacity (4,096 candidates of 32 x 32 tiles fill 27.7 of an
// SM's 32 warp slots) then spreads over the SMs in steps of four warps, not
// eight, so no SM carries many more candidates than the others.
constexpr int kSimThreads = 128;

template <int M, int NS>
void occupancy_of(int *blocks, size_t smem) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, sim_kernel<M, NS, false>, kSimThreads, smem);
}

template <int M, int NS>
void set_smem_attr(size_t smem) {
    cudaFuncSetAttribute(sim_kernel<M, NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(sim_kernel<M, NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (M > 1)
        cudaFuncSetAttribute(sim_kernel<M, NS, true, false, (M > 1)>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
}

template <int M, int NS>
void launch_one(bool gen, bool cap, unsigned blocks, int threads, size_t smem, cudaStream_t stream,
                const DevPlatform &dp, const KArgs &a, unsigned long long *ctr) {
    if (cap && M > 1) sim_kernel<M, NS, true, false, (M > 1)><<<blocks, threads, smem, stream>>>(dp, a, ctr);
    else if (gen) sim_kernel<M, NS, true><<<blocks, threads, smem, stream>>>(dp, a, ctr);
    else sim_kernel<M, NS, false><<<blocks, threads, smem, stream>>>(dp, a, ctr);
}

// Table-1 metrics of simulated schedules, one warp per candidate: the tasks'
// summed execution time (finish - start), the task count, the summed block
// size of the tasks (each base task at level l holds c_cnt[op][l] tasks of
// block b >> l), and the hierarchy depth 1 + max level.
__global__ void metrics_kernel(const hesp_cand *cands, const int8_t *levels, int64_t n_cand, const int64_t *sched_off,
                               const int64_t *start, const int64_t *finish, int64_t *busy, int64_t *ntasks,
                               int64_t *sum_block, int32_t *depth) {
    __shared__ DecodeTables s_tab;
    load_tables(s_tab);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= n_cand) return;
    const hesp_cand cd = cands[c];
    const int n = cd.n_tiles, b = cd.b;
    const int64_t nb = (int64_t)n * (n + 1) * (n + 2) / 6;
    int64_t cnt = 0, sb = 0;
    int lmax = 0;
    for (int64_t t = lane; t < nb; t += 32) {
        int op, K, I, J;
        decode_base(n, t, op, K, I, J);
        const int l = levels[cd.level_offset + t];
        cnt += s_tab.cnt[op][l];
        sb += (int64_t)s_tab.cnt[op][l] * (b >> l);
        lmax = max(lmax, l);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        cnt += __shfl_xor_sync(FULL, cnt, o);
        sb += __shfl_xor_sync(FULL, sb, o);
    }
    lmax = __reduce_max_sync(FULL, lmax);
    int64_t bz = 0;
    if (sched_off) {
        const int64_t o0 = sched_off[c];
        for (int64_t j = lane; j < cnt; j += 32) bz += finish[o0 + j] - start[o0 + j];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) bz += __shfl_xor_sync(FULL, bz, o);
    }
    if (lane == 0) {
        if (busy) busy[c] = sched_off ? bz : -1;
        if (ntasks) ntasks[c] = cnt;
        if (sum_block) sum_block[c] = sb;
        if (depth) depth[c] = 1 + lmax;
    }
}

}  // namespace

int launch_metrics(const hesp_cand *cands, const int8_t *levels, int64_t n_cand, const int64_t *sched_off,
                   const int64_t *start, const int64_t *finish, int64_t *busy, int64_t *ntasks, int64_t *sum_block,
                   int32_t *depth, cudaStream_t stream) {
    if (n_cand == 0) return HESP_OK;
    const int64_t blocks = (n_cand * 32 + 255) / 256;
    metrics_kernel<<<(unsigned)blocks, 256, 0, stream>>>(cands, levels, n_cand, sched_off, start, finish, busy, ntasks,
                                                        sum_block, depth);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

// The build-only launch: expansion, dependences and successor lists of every
// candidate, kept in its own arena (dag_mode 1), no simulation.
int launch_build(const Arena &ar, const hesp_cand *cands, const int8_t *levels, int64_t n_cand, int32_t max_tiles,
                 int32_t max_level, int64_t *ntasks, int32_t *status, uint64_t layout_sig, char *ws,
                 cudaStream_t stream) {
    KArgs a;
    memset(&a, 0, sizeof a);
    a.cands = cands;
    a.levels = levels;
    a.n_cand = n_cand;
    a.max_tiles = max_tiles;
    a.max_level = max_level;
    a.status = status;
    a.ntasks = ntasks;
    a.dag_mode = 1;
    a.layout_sig = layout_sig;
    a.ar = ar;
    a.ws = ws + kWsHeaderBytes;
    a.bm_smem_words = 0;
    DevPlatform dp;
    memset(&dp, 0, sizeof dp);
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sim_kernel<1, 1, false, true>, 256, 0) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return HESP_ERR_CUDA;
    int64_t warps = (int64_t)per_sm * sms * 8;
    if (warps > n_cand) warps = n_cand;
    a.n_slots = warps;
    unsigned long long *ctr = &((WsHeader *)ws)->work_counter;
    if (cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), stream) != cudaSuccess) return HESP_ERR_CUDA;
    sim_kernel<1, 1, false, true><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, stream>>>(dp, a, ctr);
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

// Shared-memory bitmap words per warp for a workspace sized for Tcap tasks
// (0 = the bitmap stays in the arena): up to 2048 words (64 Ki tasks).
int sim_bitmap_smem_words(int64_t Tcap) {
    const int64_t w = (Tcap + 31) / 32;
    return w <= 2048 ? (int)w : 0;
}

int sim_kernel_occupancy(int n_mem, int n_procs, int64_t Tcap, int *blocks_per_sm, int *threads_per_block) {
    *threads_per_block = kSimThreads;
    const size_t smem = (size_t)sim_bitmap_smem_words(Tcap) * 4 * (kSimThreads / 32);
    const bool two = n_procs > 32;
    switch (n_mem) {
    case 1: two ? set_smem_attr<1, 2>(smem) : set_smem_attr<1, 1>(smem); break;
    case 2: two ? set_smem_attr<2, 2>(smem) : set_smem_attr<2, 1>(smem); break;
    case 3: two ? set_smem_attr<3, 2>(smem) : set_smem_attr<3, 1>(smem); break;
    case 4: two ? set_smem_attr<4, 2>(smem) : set_smem_attr<4, 1>(smem); break;
    default: return HESP_ERR_ARG;
    }
    switch (n_mem) {
    case 1: two ? occupancy_of<1, 2>(blocks_per_sm, smem) : occupancy_of<1, 1>(blocks_per_sm, smem); break;
    case 2: two ? occupancy_of<2, 2>(blocks_per_sm, smem) : occupancy_of<2, 1>(blocks_per_sm, smem); break;
    case 3: two ? occupancy_of<3, 2>(blocks_per_sm, smem) : occupancy_of<3, 1>(blocks_per_sm, smem); break;
    case 4: two ? occupancy_of<4, 2>(blocks_per_sm, smem) : occupancy_of<4, 1>(blocks_per_sm, smem); break;
    }
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

int launch_sim(const hesp_platform *p, const DevPlatform &dp, const Arena &ar, int64_t n_slots,
               const hesp_cand *cands, const int8_t *levels, int64_t n_cand, int32_t max_tiles, int32_t max_level,
               int64_t *makespan, int32_t *status, int64_t *ntasks, const int64_t *sched_off, int16_t *sproc,
               int64_t *sstart, int64_t *sfinish, int8_t *crit, int dag_mode, uint64_t layout_sig, int fmode,
               int32_t fm_b, char *ws,
               cudaStream_t stream) {
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
    a.crit = crit;
    a.dag_mode = dag_mode;
    a.layout_sig = layout_sig;
    a.fmode = fmode;
    a.fm_b = fm_b;
    a.ar = ar;
    a.n_slots = n_slots;
    a.ws = ws + kWsHeaderBytes;
    a.bm_smem_words = p->tune_bitmap == 1 ? 0 : sim_bitmap_smem_words(ar.Tcap);
    unsigned long long *ctr = &((WsHeader *)ws)->work_counter;
    if (cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), stream) != cudaSuccess) return HESP_ERR_CUDA;
    const int threads = kSimThreads;
    const size_t smem = (size_t)a.bm_smem_words * 4 * (threads / 32);
    const int64_t blocks = (n_slots * 32 + threads - 1) / threads;
    const bool two = p->n_procs > 32;
    const unsigned ub = (unsigned)blocks;
    const bool gen = p->order != HESP_ORDER_FCFS || p->select != HESP_SELECT_EFT || p->cache != HESP_CACHE_WB ||
                     p->use_links || crit != nullptr || fmode != 0 || p->use_cap;
    const bool cap = p->use_cap && fmode == 0;
    switch (p->n_mem) {
    case 1: two ? launch_one<1, 2>(gen, cap, ub, threads, smem, stream, dp, a, ctr)
                : launch_one<1, 1>(gen, cap, ub, threads, smem, stream, dp, a, ctr); break;
    case 2: two ? launch_one<2, 2>(gen, cap, ub, threads, smem, stream, dp, a, ctr)
                : launch_one<2, 1>(gen, cap, ub, threads, smem, stream, dp, a, ctr); break;
    case 3: two ? launch_one<3, 2>(gen, cap, ub, threads, smem, stream, dp, a, ctr)
                : launch_one<3, 1>(gen, cap, ub, threads, smem, stream, dp, a, ctr); break;
    case 4: two ? launch_one<4, 2>(gen, cap, ub, threads, smem, stream, dp, a, ctr)
                : launch_one<4, 1>(gen, cap, ub, threads, smem, stream, dp, a, ctr); break;
    default:
        return HESP_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

}  // namespace hesp
