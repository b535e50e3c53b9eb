// Internal declarations shared by the CUDA sources of libhesp.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hesp.h"

#define HESP_LB (HESP_MAX_LOG2_BLOCK + 1)  // exec table entries per (op, type): block 2^0 .. 2^20

struct hesp_platform {
    int32_t n_mem, n_types, n_procs;
    int64_t xfer_latency_ns, bytes_per_elem, bw_bytes_per_ns;
    hesp_ptype types[HESP_MAX_TYPES];
    hesp_proc procs[HESP_MAX_PROCS];
    // exec[op][type][log2 block] in ns; -1 where the model does not fit in
    // 56 bits (the simulator then flags the candidate with HESP_ERR_ARG).
    int64_t exec[4][HESP_MAX_TYPES][HESP_LB];
    // launch shape chosen by hesp_sim_autotune or set by the caller (0 = default)
    int32_t tune_ctas_per_sm;
    int32_t tune_bitmap;  // 0 auto, 1 arena (global memory), 2 shared memory when it fits
    // scheduling heuristics (Sec. 2.1): task order 0 FCFS / 1 PL, processor
    // choice 0 EFT-P / 1 EIT-P / 2 F-P / 3 R-P, and the seed of R-P's draws
    int32_t order, select;
    uint64_t rp_seed;
    int32_t cache;  // 0 write-back, 1 write-through, 2 write-around
    // network topology: with use_links, a message s -> d takes
    // link_lat[s][d] + ceil(bytes / link_bw[s][d]) ns
    int32_t use_links;
    int64_t link_lat[HESP_MAX_MEMS][HESP_MAX_MEMS], link_bw[HESP_MAX_MEMS][HESP_MAX_MEMS];
    // finite accelerator memories: capacity in bytes per memory (0 = unbounded)
    int32_t use_cap;
    int64_t cap_bytes[HESP_MAX_MEMS];
};

struct hesp_dag {
    int32_t n_tiles, b, max_level;
    int64_t n_base;
    int32_t *op, *k, *i, *j;  // host arrays of n_base
};

namespace hesp {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter-based generator:
// value k of stream c is the published output function applied to
// seed + ((c << 32) + k + 1) * 0x9E3779B97F4A7C15; a draw in [0, m) is
// Lemire's multiply-shift ((u >> 32) * m) >> 32.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t sm64_at(uint64_t seed, uint64_t c, uint64_t k) {
    return sm64_mix(seed + ((c << 32) + k + 1) * kGamma);
}

__device__ __forceinline__ uint32_t lemire_draw(uint64_t u, uint32_t m) { return (uint32_t)(((u >> 32) * m) >> 32); }

// Platform image passed by value to the simulation kernel (constant bank),
// copied to shared memory at kernel start.
struct DevPlatform {
    int32_t n_mem, n_types, n_procs, pad;
    int32_t order, select;  // task order (0 FCFS, 1 PL) and processor choice (0 EFT-P, 1 EIT-P, 2 F-P, 3 R-P)
    uint64_t rp_seed;       // R-P: seed of the per-task draws
    int32_t cache, use_links;  // caching policy (0 WB, 1 WT, 2 WA); per-link transfer costs
    int64_t link_lat[HESP_MAX_MEMS * HESP_MAX_MEMS], link_bw[HESP_MAX_MEMS * HESP_MAX_MEMS];
    int32_t use_cap, pad2;  // finite accelerator memories
    int64_t cap_bytes[HESP_MAX_MEMS];
    int64_t exec[4 * HESP_MAX_TYPES * HESP_LB];
    int64_t wsum[4 * HESP_LB];  // task time summed over all processors, per (op, log2 block); -1 if any is -1
    int8_t proc_mem[HESP_MAX_PROCS];
    int8_t proc_type[HESP_MAX_PROCS];
    int64_t lat, bpe, bw;
};

// Per-warp arena of the simulator (one arena per concurrently simulated
// candidate).  Capacities hold any candidate with n <= max_tiles and
// levels <= max_level; offsets are bytes from the arena start.
struct Arena {
    int64_t slot_bytes;
    int64_t Tcap;  // tasks
    int64_t Ecap;  // dependence edges
    int64_t Acap;  // atoms
    int64_t Kcap;  // transfer-table entries (atoms per task + 1)
    // The edge list of the dependence build (epred: the predecessor of each
    // edge, grouped by successor) lives in the FIFO link area and the
    // per-task marks in the successor offsets: neither is in use at the same
    // time as what it shares memory with.
    int64_t off_desc, off_pending, off_link, off_next, off_succoff, off_succ, off_epred, off_lw, off_vfrom,
        off_bitmap, off_xt, off_hist, off_pend0, off_hdr, off_use;
};

// Optional areas of an arena (the `room` flags of make_arena): a launch
// only touches the areas its platform and mode need, so a workspace sized
// without them holds more concurrent candidates.
constexpr unsigned kRoomPL = 1;    // priority-list order: 32 bytes per task in the link area (else 16)
constexpr unsigned kRoomKept = 2;  // keep / reuse: the initial pending counts and the candidate header
constexpr unsigned kRoomCap = 4;   // finite memories: the last use of every atom per memory
constexpr unsigned kRoomAll = kRoomPL | kRoomKept | kRoomCap;

// Header at the start of the workspace.
struct WsHeader {
    unsigned long long work_counter;
    unsigned long long pad[31];
};
constexpr int64_t kWsHeaderBytes = 256;

// Closed forms used to size arenas (host side).
int64_t tasks_uniform(int64_t n, int level);  // tasks when every base task is split `level` times
int64_t regions_uniform(int64_t n, int level); // sum over those tasks of their region count
Arena make_arena(int32_t max_tiles, int32_t max_level, int32_t n_mem, int64_t task_cap, unsigned room);
Arena make_arena_factors(int32_t max_tiles, int32_t max_factor, int32_t n_mem, int64_t task_cap, unsigned room);
unsigned arena_room_of(const hesp_platform *p);  // the optional areas a platform's launches use

int sim_slots_for(const hesp_platform *p, const Arena &ar, int64_t *resident_warps);  // device resident warps
int launch_sim(const hesp_platform *p, const DevPlatform &dp, const Arena &ar, int64_t n_slots,
               const hesp_cand *cands, const int8_t *levels, int64_t n_cand, int32_t max_tiles, int32_t max_level,
               int64_t *makespan, int32_t *status, int64_t *ntasks, const int64_t *sched_off, int16_t *sproc,
               int64_t *sstart, int64_t *sfinish, int8_t *crit, int dag_mode, uint64_t layout_sig, int fmode,
               int32_t fm_b, char *ws,
               cudaStream_t stream);
int sim_kernel_occupancy(int n_mem, int n_procs, int64_t Tcap, int *blocks_per_sm, int *threads_per_block);
int launch_build(const Arena &ar, const hesp_cand *cands, const int8_t *levels, int64_t n_cand, int32_t max_tiles,
                 int32_t max_level, int64_t *ntasks, int32_t *status, uint64_t layout_sig, char *ws,
                 cudaStream_t stream);
int launch_metrics(const hesp_cand *cands, const int8_t *levels, int64_t n_cand, const int64_t *sched_off,
                   const int64_t *start, const int64_t *finish, int64_t *busy, int64_t *ntasks, int64_t *sum_block,
                   int32_t *depth, cudaStream_t stream);
int sim_bitmap_smem_words(int64_t Tcap);

int launch_generate(int32_t kind, uint64_t seed, int64_t first, int64_t n_cand, int32_t n_tiles, int32_t b,
                    int32_t n_levels, hesp_cand *cands, int8_t *levels, cudaStream_t stream);
int launch_mutate(const int8_t *parents, int32_t n_parents, int32_t n_base, int32_t n_levels, uint32_t p_num,
                  uint64_t seed, int64_t first, int64_t n, int8_t *out, cudaStream_t stream);
int launch_sort_by_size(const hesp_cand *in, const int8_t *levels, int64_t n, hesp_cand *out, int32_t *perm,
                        void *ws, cudaStream_t st);
int launch_generate_uneven(uint64_t seed, int64_t first, int64_t n_cand, hesp_cand *cands, int8_t *levels,
                           int64_t levels_cap, int64_t *levels_used, cudaStream_t stream);

// Arguments of the tensor-core GEMM C = A B^T and its epilogues
// (0: fp32 C; 1: bf16 relu(acc + bias) (+ transposed); 2: bf16 acc masked by mask > 0 (+ transposed)).
struct GemmArgs {
    int M, N, K;
    int epi;
    float *C;
    int ldc;
    const float *bias;
    __nv_bfloat16 *out;
    int ldo;
    __nv_bfloat16 *out_t;
    int ldt;
    const __nv_bfloat16 *mask;
    int ldm;
    int *err;
    // one-hot A operand (launch_gemm_onehot only)
    const int8_t *oh_lv = nullptr;
    int64_t oh_stride = 0;
    int oh_base = 0, oh_levels = 0;
};
int launch_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, const GemmArgs &g, cudaStream_t st);
int launch_gemm_onehot(const int8_t *levels, int64_t stride, int n_base, int NL, const void *B, int64_t ldb,
                       const GemmArgs &g, cudaStream_t st);

}  // namespace hesp
