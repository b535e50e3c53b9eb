/*
 * hesp.h -- C ABI of libhesp.so, a single-GPU (NVIDIA B300, sm_103a) engine
 * for the data-parallel hot path of HeSP (Rey, Igual, Prieto-Matias, "HeSP: a
 * simulation framework for solving the task scheduling-partitioning problem
 * on heterogeneous architectures", arXiv 1602.05510): batched evaluation of
 * candidate partitions of the tiled Cholesky task DAG.
 *
 * Conventions
 *   - Every call returns an int status: HESP_OK (0) or a negative HESP_ERR_*.
 *     hesp_status_string() names it.
 *   - "_dev" pointers are device memory owned by the caller; "_host" pointers
 *     are host memory owned by the caller.  Opaque handles are created and
 *     destroyed by the library.
 *   - Calls that take `void* stream` (a cudaStream_t; NULL = legacy default
 *     stream) are asynchronous on that stream; their per-candidate results
 *     (status words) are valid once the stream has reached them.  Argument
 *     errors are reported synchronously by the return value.
 *   - Simulated time is int64 nanoseconds.  No floating point is used in the
 *     simulation; results are exactly those of the rules described below.
 *   - Handles are not thread-safe; distinct handles may be used concurrently.
 *   - There is no CPU fallback: without a usable CUDA device the calls that
 *     launch work return HESP_ERR_CUDA.
 */
#ifndef HESP_H
#define HESP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define HESP_OK 0
#define HESP_ERR_ARG (-1)         /* invalid argument (host) or candidate (device) */
#define HESP_ERR_CAPACITY (-2)    /* a candidate exceeds the workspace capacities */
#define HESP_ERR_CUDA (-3)        /* CUDA runtime error or no device */
#define HESP_ERR_TIMEOUT (-4)     /* a candidate's event loop exceeded its iteration cap */
#define HESP_ERR_STATE (-5)       /* internal consistency check failed */
#define HESP_ERR_UNSUPPORTED (-6) /* outside the supported limits below */

const char *hesp_status_string(int status);

/* ----------------------------------------------------------------- limits */
#define HESP_MAX_MEMS 4   /* memory spaces (0 = host) */
#define HESP_MAX_TYPES 4  /* processor types */
#define HESP_MAX_PROCS 64 /* processors */
#define HESP_MAX_LEVEL 4  /* split levels per base task: 0..4 */
#define HESP_MAX_TILES 64 /* tiles per matrix side */
#define HESP_MAX_LOG2_BLOCK 20 /* block sizes are powers of two up to 2^20 */
#define HESP_MAX_FACTOR 4  /* partition factors k (p = 1/k) of hesp_simulate_factors: 1..4 */

/* Operations of the blocked Cholesky factorization (Sec. 1.1, Fig. 1). */
#define HESP_OP_CHOL 0
#define HESP_OP_TRSM 1
#define HESP_OP_SYRK 2
#define HESP_OP_GEMM 3

/* -------------------------------------------------------------- platform
 * Sec. 2: a platform is a set of memory spaces connected by a network and a
 * set of processors, each tied to one memory space; Sec. 2.1 "Performance and
 * data transfer models": task and transfer times come from models given a
 * priori.
 *
 * Processor type model: a task of operation op on a bs x bs block takes
 *     ceil(flops / rate) ns,  flops = {1, 3, 3, 6}[op] * bs^3 / 3,
 *     rate = peak_gflops * eff_pct[op] / 100 * bs^2 / (bs^2 + h^2) GFLOP/s,
 * unless overridden by hesp_platform_set_exec_table (measured models).
 * Transfer model (every pair of memories, no contention): a message of E
 * elements takes xfer_latency_ns + ceil(bytes_per_elem * E / bw_bytes_per_ns).
 * Memory 0 is host memory; accelerator memories act as write-back software
 * caches of it (Sec. 2.1).  Memories have unlimited capacity. */
typedef struct {
    int64_t peak_gflops;
    int64_t h;
    int32_t eff_pct[4]; /* indexed by HESP_OP_* */
} hesp_ptype;

typedef struct {
    int32_t memory; /* 0 .. n_mem-1 */
    int32_t type;   /* 0 .. n_types-1 */
} hesp_proc;

typedef struct {
    int32_t n_mem;          /* 1 .. HESP_MAX_MEMS */
    int32_t n_types;        /* 1 .. HESP_MAX_TYPES */
    const hesp_ptype *types;
    int32_t n_procs;        /* 1 .. HESP_MAX_PROCS; processor id = index */
    const hesp_proc *procs;
    int64_t xfer_latency_ns;
    int64_t bytes_per_elem;
    int64_t bw_bytes_per_ns; /* >= 1 when n_mem > 1 */
} hesp_platform_desc;

typedef struct hesp_platform hesp_platform;

/* Copies `desc` (host memory) into a new handle.  ERR_ARG on invalid fields,
 * ERR_UNSUPPORTED beyond the limits. */
int hesp_platform_create(const hesp_platform_desc *desc, hesp_platform **out);
/* Override the time of (op, type, block) with `ns` (a measured model,
 * Sec. 2.1 / Sec. 3).  `block` must be a power of two <= 2^20, ns >= 1. */
int hesp_platform_set_exec_table(hesp_platform *p, int32_t op, int32_t type, int64_t block, int64_t ns);
/* Scheduling heuristics of Sec. 2.1 used when simulating on this platform.
 * Task order:
 *   HESP_ORDER_FCFS (0, default): at each event time the released tasks join
 *   a first-come first-served queue in ascending id and are scheduled from
 *   its front;
 *   HESP_ORDER_PL (1): a priority list (HEFT-like) -- critical time of a task
 *   = its time summed over all processors (the mean times P) plus the largest
 *   critical time among its successors; tasks are scheduled in decreasing
 *   critical time (ties: lower id), each at its release time (the latest
 *   finish among its predecessors).
 * Processor choice (ties to the lowest processor id):
 *   HESP_SELECT_EFT (0, default): earliest finish time including transfers;
 *   HESP_SELECT_EIT (1): the processor that becomes idle first, max(t, avail);
 *   HESP_SELECT_FP (2): the fastest for the task among the processors idle at
 *   the scheduling time t (nothing running or queued on them after t);
 *   HESP_SELECT_RP (3): among the processors idle at t, in id order, the one
 *   at index ((u >> 32) * n_idle) >> 32, u = SplitMix64 output for counter
 *   (c = task id, k = 0) under rp_seed (Steele et al. 2014, Lemire's draw).
 *   Under F-P and R-P a task waits while no processor is idle: in FCFS order
 *   the queue waits for the next completion; in PL order the task is
 *   scheduled when the first processor becomes idle.
 * rp_seed is used by R-P only.  ERR_ARG for an unknown order or choice. */
#define HESP_ORDER_FCFS 0
#define HESP_ORDER_PL 1
#define HESP_SELECT_EFT 0
#define HESP_SELECT_EIT 1
#define HESP_SELECT_FP 2
#define HESP_SELECT_RP 3
int hesp_platform_set_policy(hesp_platform *p, int32_t order, int32_t select, uint64_t rp_seed);
/* Caching of accelerator memories (Sec. 2.1), applied to the block a task
 * writes (every other copy of it is invalidated):
 *   HESP_CACHE_WB (0, default): write-back -- valid only in the memory of the
 *   task's processor, from its finish;
 *   HESP_CACHE_WT (1): write-through -- also sent to host memory at the
 *   finish: valid there from finish + xfer(block elements);
 *   HESP_CACHE_WA (2): write-around -- when the processor is not in host
 *   memory, valid only in host memory, from finish + xfer(block elements).
 * A fetch of data that no memory can supply at the scheduling time t (under
 * WT / WA a copy may still be in flight to the host) takes the copy usable
 * first (ties to the lower memory); one message per source memory, issued at
 * t or, if later, when the last of its data is usable there.  ERR_ARG for an
 * unknown policy. */
#define HESP_CACHE_WB 0
#define HESP_CACHE_WT 1
#define HESP_CACHE_WA 2
int hesp_platform_set_cache(hesp_platform *p, int32_t cache);
/* Network topology (Sec. 2): a direct link per ordered pair of memories.
 * After this call a message from memory src to memory dst of E elements
 * takes latency_ns + ceil(E * bytes_per_elem / bw_bytes_per_ns) ns; pairs
 * never set keep the platform's xfer_latency_ns / bw_bytes_per_ns.  Links
 * carry any number of messages at once (no contention).  ERR_ARG for src ==
 * dst, a memory out of range, latency < 0 or bandwidth < 1. */
int hesp_platform_set_link(hesp_platform *p, int32_t src, int32_t dst, int64_t latency_ns, int64_t bw_bytes_per_ns);

/* Finite memory spaces (Sec. 2: a platform of "finite-size memory spaces";
 * the paper gives no eviction policy, so this is a reading).  Memory `mem`
 * (an accelerator memory, 1 .. n_mem - 1; host memory is unbounded) holds at
 * most `bytes` bytes of data, counted in whole atoms (the blocks of side
 * b / 2^L of a candidate whose deepest split level is L); 0 = unbounded (the
 * default).  When task j is scheduled at time t, a finite memory m can take
 * it when the atoms j lacks in m fit in m's free space plus the atoms m may
 * evict -- valid in m, not used by j, and not used by a task in flight on a
 * processor of m (the latest finish of a task that used the atom there is
 * <= t); processors of memories that cannot take j are not candidates, and
 * a task no memory can take gives its candidate HESP_ERR_CAPACITY.  On the
 * chosen memory, atoms are evicted least recently used first (that latest
 * finish, ties to the lower atom index) until j's atoms fit; evicted atoms
 * valid in no other memory are written back to host memory, in one message
 * issued at t, and are valid there from its arrival.  Supported with EFT-P
 * and EIT-P (hesp_simulate_batch returns HESP_ERR_ARG under F-P / R-P) and
 * dyadic partitions (hesp_simulate_factors returns HESP_ERR_UNSUPPORTED);
 * every task order and caching policy.  Returns HESP_ERR_ARG for a bad
 * memory or a negative size. */
int hesp_platform_set_capacity(hesp_platform *p, int32_t mem, int64_t bytes);
/* Host queries of the models, as used by the simulator. */
int hesp_platform_exec_ns(const hesp_platform *p, int32_t op, int32_t type, int64_t block, int64_t *ns_out);
int hesp_platform_xfer_ns(const hesp_platform *p, int64_t elems, int64_t *ns_out);
void hesp_platform_destroy(hesp_platform *p);

/* ------------------------------------------------------------------- DAG
 * Sec. 1.1 Fig. 1: the base tasks of an n x n tiled Cholesky (upper storage,
 * A[k][j], j >= k) in the loop order
 *     for k: chol(k); for j>k: trsm(k,j); for i>k: { for j>i: gemm(k,i,j); syrk(k,i) }
 * Sec. 2.1 "Recursive task partitioners": a base task with split level l is
 * replaced in place by the tasks of its 2x2 blocked algorithm, recursively l
 * times (chol -> 4, trsm -> 6, syrk -> 6, gemm -> 8 tasks per level); task
 * ids follow the depth-first order of this expansion. */
typedef struct hesp_dag hesp_dag;

int hesp_dag_build(int32_t n_tiles, int32_t b, int32_t max_level, hesp_dag **out);
int64_t hesp_dag_n_base(const hesp_dag *d);
/* Base task list (host arrays of hesp_dag_n_base entries): op and tile
 * indices (k, i, j) with chol(k): i = j = k; trsm(k, j): i = k; syrk(k, i): j = i. */
int hesp_dag_base_tasks(const hesp_dag *d, int32_t *op_host, int32_t *k_host, int32_t *i_host, int32_t *j_host);
/* Tasks of one partition vector (levels_host: n_base int8 in 0..max_level),
 * and the flop total times 3 (must equal (n b)^3 for every partition). */
int hesp_dag_count_tasks(const hesp_dag *d, const int8_t *levels_host, int64_t *n_tasks_out,
                         int64_t *flops3_out);
void hesp_dag_destroy(hesp_dag *d);

/* ---------------------------------------------------- batched simulation
 * One candidate = (n_tiles, b, levels[level_offset .. + n_base)).  b must be
 * a power of two with b >> max(levels) >= 1. */
typedef struct {
    int32_t n_tiles;
    int32_t b;
    int64_t level_offset;
} hesp_cand;

/* Bytes of device workspace needed to simulate candidates with at most
 * `max_tiles` tiles and split levels <= `max_level` on platform `p`, using up
 * to `n_cand` concurrent candidates (the library caps it at the number of
 * resident warps of the current device).  task_cap = 0 sizes each candidate's
 * arena for the largest DAG these bounds allow; task_cap > 0 sizes it for
 * that many tasks (and 4 dependence edges per task), and candidates that do
 * not fit get HESP_ERR_CAPACITY.  The workspace is caller-owned device
 * memory, 256-byte aligned, reused across calls on one stream. */
int hesp_sim_workspace_size(const hesp_platform *p, int32_t max_tiles, int32_t max_level, int64_t task_cap,
                            int64_t n_cand, size_t *bytes_out);

/* Simulate n_cand candidates (HeSP Sec. 2.1: the platform's task order and
 * processor selection, hesp_platform_set_policy -- by default FCFS at release
 * time and EFT-P -- with write-back caching and prefetching transfers).
 * For each candidate: expand its DAG, derive RaW/WaW/WaR dependences from the
 * overlap of the tasks' data blocks, then run the event loop (FCFS):
 *   t = 0; released = tasks without predecessors; repeat: schedule every
 *   released task in ascending id at time t; t = earliest finish in flight;
 *   complete every task finishing at t; released = tasks whose predecessors
 *   all completed.
 * Scheduling task j at time t: for each memory m, DRT(j, m) = latest of the
 * times its data is usable in m -- a copy valid in m is usable from the time
 * it was written or arrived; data valid nowhere usable in m is fetched from
 * the lowest-numbered memory holding a copy usable at t, one message per
 * source memory issued at t.  EFT(p) = max(t, avail(p), DRT(j, mem(p))) +
 * exec(op, type(p), block); the processor with the smallest EFT wins, ties to
 * the lowest id.  Fetched data becomes valid in the chosen memory from its
 * arrival; the written block then becomes valid only there, from the finish
 * time.  The makespan is the largest finish time.
 *
 * Inputs (device): cands_dev[n_cand], levels_dev (int8, addressed through
 * level_offset).  max_tiles / max_level / task_cap bound every candidate and
 * must match the workspace sizing.
 * Outputs (device): makespan_dev[n_cand] (-1 on error), status_dev[n_cand]
 * (HESP_OK or HESP_ERR_ARG / _CAPACITY / _TIMEOUT / _STATE for that
 * candidate), ntasks_dev[n_cand] (nullable: task count of each candidate).
 * Optional schedule (all four non-NULL or all NULL): task j of candidate c is
 * written at index sched_offsets_dev[c] + j of proc_dev (int16 processor id),
 * start_dev and finish_dev (int64 ns); the caller sizes them with
 * hesp_dag_count_tasks.
 * workspace: from hesp_sim_workspace_size for the same platform, max_tiles,
 * max_level; any size >= the size for n_cand = 1 works (fewer candidates then
 * run concurrently). */
int hesp_simulate_batch(const hesp_platform *p, const hesp_cand *cands_dev, const int8_t *levels_dev,
                        int64_t n_cand, int32_t max_tiles, int32_t max_level, int64_t task_cap,
                        int64_t *makespan_dev, int32_t *status_dev, int64_t *ntasks_dev, const int64_t *sched_offsets_dev,
                        int16_t *proc_dev, int64_t *start_dev, int64_t *finish_dev, void *workspace_dev,
                        size_t workspace_bytes, void *stream);

/* General partition parameter (Sec. 2.1, "Iterative solver": a partition
 * cuts a task's blocks of size d into blocks of size p d, p in (0, 1]; Fig. 4:
 * partially overlapping blocks of two tilings of one block).  Each base task
 * t of the Fig. 1 loop is cut once with p = 1 / k, k = factors[t] in
 * 1 .. max_factor (k = 1 keeps it): it is replaced by its k-way blocked
 * algorithm, whose tasks are not cut again --
 *   chol(A):   the Fig. 1 loop on the k x k blocks of A;
 *   trsm(T,B): B := T^-T B, for p: { for c: trsm(Tpp -> Bpc);
 *              for i > p: for c: gemm(Tpi, Bpc -> Bic) };
 *   syrk(A,C): for p: for i: { for j > i: gemm(Api, Apj -> Cij); syrk(Api -> Cii) };
 *   gemm(A,B,C): for p, i, j: gemm(Api, Bpj -> Cij).
 * k = 2 is the 2x2 partition of hesp_simulate_batch at level 1 (the same
 * tasks in the same order); mixing k = 2 and 3 on one tile gives the
 * non-dyadic tilings of Fig. 4.  Dependences and coherence are tracked on
 * the common refinement of all the tilings: atoms of side b / L, L the least
 * common multiple of the candidate's factors (b must be a multiple of L).
 * Task times: exec(op, type, b / k) from the platform's table where b / k is
 * a power of two (so hesp_platform_set_exec_table applies), else from the
 * performance model of hesp_ptype.  The simulation itself (policies,
 * caching, links, event loop, outputs) is that of hesp_simulate_batch.
 *
 * Inputs (device): cands_dev[n_cand] (n_tiles <= max_tiles; b must equal
 * the argument b, else the candidate gets HESP_ERR_ARG), factors_dev (int8,
 * one factor per base task, addressed through level_offset).  max_factor
 * (1 .. HESP_MAX_FACTOR) and task_cap bound every candidate and must match
 * the workspace sizing (hesp_sim_workspace_size_factors; the arena holds up
 * to 16 dependence edges per task, more give HESP_ERR_CAPACITY).  Outputs
 * and the optional schedule as for hesp_simulate_batch (the schedule's
 * sizes: the task counts of the k-way partitions, e.g. from ntasks_dev of a
 * first call).  crit_dev (nullable, int8, addressed like factors_dev):
 * the critical-path flags of hesp_simulate_critical, per base task, for the
 * iterative solver over factors.  Returns HESP_ERR_UNSUPPORTED for max_factor or max_tiles
 * outside the limits, HESP_ERR_ARG for bad pointers or sizes; asynchronous
 * on `stream`. */
int hesp_sim_workspace_size_factors(const hesp_platform *p, int32_t max_tiles, int32_t max_factor, int64_t task_cap,
                                    int64_t n_cand, size_t *bytes_out);
int hesp_simulate_factors(const hesp_platform *p, const hesp_cand *cands_dev, const int8_t *factors_dev,
                          int64_t n_cand, int32_t max_tiles, int32_t max_factor, int32_t b, int64_t task_cap,
                          int64_t *makespan_dev, int32_t *status_dev, int64_t *ntasks_dev,
                          const int64_t *sched_offsets_dev, int16_t *proc_dev, int64_t *start_dev,
                          int64_t *finish_dev, int8_t *crit_dev, void *workspace_dev, size_t workspace_bytes,
                          void *stream);

/* Table 1 metrics (Sec. 3) of simulated candidates, one value per candidate:
 *   busy_dev[c]      = sum over its tasks of finish - start (the processors'
 *                      total busy time; average load = busy / (P * makespan));
 *                      -1 when no schedule is given;
 *   ntasks_dev[c]    = its task count;
 *   sum_block_dev[c] = sum over its tasks of the block size (average block
 *                      size = sum_block / ntasks);
 *   depth_dev[c]     = 1 + its deepest split level (the levels of its task
 *                      hierarchy).
 * GFLOPS = (n b)^3 / 3 / makespan.  Inputs as for hesp_simulate_batch; the
 * schedule (sched_offsets_dev, start_dev, finish_dev: all three or none) is
 * the one hesp_simulate_batch wrote.  Any output pointer may be NULL.  All
 * device pointers; asynchronous on `stream`. */
int hesp_schedule_metrics(const hesp_cand *cands_dev, const int8_t *levels_dev, int64_t n_cand,
                          const int64_t *sched_offsets_dev, const int64_t *start_dev, const int64_t *finish_dev,
                          int64_t *busy_dev, int64_t *ntasks_dev, int64_t *sum_block_dev, int32_t *depth_dev,
                          void *stream);

/* Several platforms, one DAG build.  A candidate's DAG (tasks, dependences)
 * depends only on its partition, so simulating the same candidates on
 * several platforms (or scheduling policies) need not expand and analyse
 * them again: hesp_simulate_batch_keep simulates like hesp_simulate_batch
 * and keeps each candidate's DAG in its own arena of the workspace;
 * hesp_simulate_batch_reuse then simulates the candidates on another
 * platform from the kept DAGs.  Results equal hesp_simulate_batch's.
 *   - The workspace holds one arena per candidate (n_cand arenas, laid out
 *     for HESP_MAX_MEMS memories whatever the platform): size it with
 *     hesp_sim_workspace_size_kept; ERR_ARG if it is smaller.
 *   - A reuse call must pass the same cands_dev (same order), levels,
 *     max_tiles, max_level and task_cap as the keep call whose DAGs are in
 *     the workspace; each arena records the layout and a hash of its
 *     candidate's (n_tiles, b, levels), and a candidate whose record does
 *     not match gets HESP_ERR_STATE (a candidate whose build failed gets the
 *     build's status).
 *   - Any number of reuse calls may follow one keep call. */
int hesp_sim_workspace_size_kept(int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t n_cand,
                                 size_t *bytes_out);
/* The DAG part of a keep call alone (no platform, no simulation): expand and
 * analyse every candidate and keep its DAG in its arena, for
 * hesp_simulate_batch_reuse calls.  status_dev[c] is the build's status
 * (HESP_OK, HESP_ERR_ARG or HESP_ERR_CAPACITY), ntasks_dev (nullable) the
 * task counts. */
int hesp_dag_build_kept(const hesp_cand *cands_dev, const int8_t *levels_dev, int64_t n_cand, int32_t max_tiles,
                        int32_t max_level, int64_t task_cap, int32_t *status_dev, int64_t *ntasks_dev,
                        void *workspace_dev, size_t workspace_bytes, void *stream);
int hesp_simulate_batch_keep(const hesp_platform *p, const hesp_cand *cands_dev, const int8_t *levels_dev,
                             int64_t n_cand, int32_t max_tiles, int32_t max_level, int64_t task_cap,
                             int64_t *makespan_dev, int32_t *status_dev, int64_t *ntasks_dev, void *workspace_dev,
                             size_t workspace_bytes, void *stream);
int hesp_simulate_batch_reuse(const hesp_platform *p, const hesp_cand *cands_dev, const int8_t *levels_dev,
                              int64_t n_cand, int32_t max_tiles, int32_t max_level, int64_t task_cap,
                              int64_t *makespan_dev, int32_t *status_dev, int64_t *ntasks_dev, void *workspace_dev,
                              size_t workspace_bytes, void *stream);

/* ------------------------------------------------ iterative partition solver
 * HeSP's iterative solver (Sec. 2.1 "Iterative solver"): each iteration is a
 * schedule stage (simulate the partition) and a partition stage (list
 * candidate moves, score them, pick one).  A partition is one split level per
 * base task; move k = 2 t + d changes base task t by +1 (d = 0, partition) or
 * -1 (d = 1, merge back).  Candidate moves, in increasing k: a partition move
 * for each base task chosen by the selection policy and below the deepest
 * level, and a merge move for every split base task (an existing task
 * cluster).  Selection: HESP_SOLVER_ALL every base task; HESP_SOLVER_CP the
 * base tasks flagged by hesp_simulate_critical; HESP_SOLVER_SHALLOW the base
 * tasks at the minimal level (depth).  A move's score is the current
 * makespan minus its simulated makespan (the paper estimates it; here the
 * whole neighbourhood is simulated in one hesp_simulate_batch call); moves
 * with a score <= 0 or a failed simulation are dropped.  Sampling:
 * HESP_PICK_HARD the largest score, ties to the lower index; HESP_PICK_SOFT
 * r = floor(u * S / 2^64) with S the sum of the kept scores and u the
 * SplitMix64 output for counter (c = iteration, k = 0) under `seed`, then the
 * first kept move whose running score sum exceeds r (probability score / S). */
#define HESP_SOLVER_ALL 0
#define HESP_SOLVER_CP 1
#define HESP_SOLVER_SHALLOW 2
#define HESP_PICK_HARD 0
#define HESP_PICK_SOFT 1

/* hesp_simulate_batch (no schedule output) that also flags, per base task,
 * whether one of its tasks lies on the critical path of the candidate's
 * schedule: the longest path of the DAG weighted by the scheduled task
 * times; a task is on it when the longest path through it is as long as the
 * longest path overall.  crit_dev (int8, device) is laid out like the levels:
 * crit_dev[level_offset + t] = 1 or 0 for base task t.  Always runs the
 * general-policy kernel.  Errors as hesp_simulate_batch. */
int hesp_simulate_critical(const hesp_platform *p, const hesp_cand *cands_dev, const int8_t *levels_dev,
                           int64_t n_cand, int32_t max_tiles, int32_t max_level, int64_t task_cap,
                           int64_t *makespan_dev, int32_t *status_dev, int8_t *crit_dev, void *workspace_dev,
                           size_t workspace_bytes, void *stream);

/* Partition stage, step (1): the candidate moves of the partition levels_dev
 * (int8[n_base], device, levels 0 .. n_levels - 1).  Writes the move codes in
 * increasing k to moves_dev (int32, capacity 2 n_base), their number to
 * *count_dev (int64, device), and, when rows_dev is not NULL, the moved
 * partitions to rows_dev (int8, row r = levels with move r applied, capacity
 * 2 n_base x n_base; rows past the count are left untouched).  crit_dev
 * (int8[n_base]) is read for HESP_SOLVER_CP only.  ERR_ARG on a bad argument,
 * ERR_UNSUPPORTED for n_base > 32767.  Asynchronous on `stream`. */
int hesp_solver_moves(const int8_t *levels_dev, int32_t n_base, int32_t n_levels, int32_t mode,
                      const int8_t *crit_dev, int32_t *moves_dev, int64_t *count_dev, int8_t *rows_dev, void *stream);

/* hesp_solver_moves over any value range [lo, hi] (0 <= lo <= hi <= 127):
 * the partition factors k of hesp_simulate_factors (lo = 1, hi = max_factor:
 * Sec. 2.1, the partition parameter p = 1/k of a task is made finer, k + 1,
 * or coarser, k - 1, down to merging the cluster back at k = 1).  A finer
 * move for each selected base task below hi, a coarser one for each base
 * task above lo; Shallow selects the base tasks at the minimal value.
 * hesp_solver_moves is this call with lo = 0, hi = n_levels - 1. */
int hesp_solver_moves_range(const int8_t *values_dev, int32_t n_base, int32_t lo, int32_t hi, int32_t mode,
                            const int8_t *crit_dev, int32_t *moves_dev, int64_t *count_dev, int8_t *rows_dev,
                            void *stream);

/* Partition stage, step (2): score the *count_dev moves from their simulated
 * makespan_dev / status_dev (index r = row r of hesp_solver_moves) against
 * *cur_makespan_dev, pick one (pick = HESP_PICK_HARD / HESP_PICK_SOFT; seed
 * and iteration drive Soft's draw), and apply it: levels_dev (the current
 * partition) and *cur_makespan_dev are updated in place and *chosen_dev is
 * the move code, or -1 when no move has a positive score (a local optimum;
 * nothing changes), or -2 when the score sum is 2^64 or more (nothing
 * changes).  All device pointers; asynchronous on `stream`. */
int hesp_solver_pick(const int64_t *makespan_dev, const int32_t *status_dev, const int32_t *moves_dev,
                     const int64_t *count_dev, int32_t pick, uint64_t seed, int64_t iteration,
                     int64_t *cur_makespan_dev, int8_t *levels_dev, int64_t *chosen_dev, void *stream);

/* Allocation-free variant of hesp_simulate_batch.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory when
 * they simulate (a memory manager that owns the whole device budget, a plugin
 * host that hands over only input and output buffers, a loop that may not
 * call cudaMalloc).  Instead of a caller workspace it uses one fixed array of
 * HESP_NOALLOC_SCRATCH_BYTES in the library's device memory, held by every
 * GPU that loads the library until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   - Arguments and results are those of hesp_simulate_batch (no workspace).
 *   - HESP_ERR_CAPACITY (synchronously) if one candidate arena for
 *     (max_tiles, max_level, platform memories) does not fit the array, e.g.
 *     max_tiles 8 / max_level 2 fits (about 180 concurrent candidates), while
 *     max_tiles 32 / max_level 3 does not.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the array and it keeps the last call's contents; each
 *     call resets what must start at zero.  Calls whose executions overlap on
 *     the GPU (different streams, or different host threads) race on it: run
 *     them one after another. */
#define HESP_NOALLOC_SCRATCH_BYTES (64u << 20)
int hesp_simulate_batch_noalloc(const hesp_platform *p, const hesp_cand *cands_dev, const int8_t *levels_dev,
                                int64_t n_cand, int32_t max_tiles, int32_t max_level, int64_t *makespan_dev,
                                int32_t *status_dev, int64_t *ntasks_dev, const int64_t *sched_offsets_dev,
                                int16_t *proc_dev, int64_t *start_dev, int64_t *finish_dev, void *stream);

/* ------------------------------------------------- runtime: graphs, tuning
 * Capture any sequence of asynchronous hesp_* calls issued on `stream` (not
 * the legacy default stream) between hesp_graph_begin and hesp_graph_end into
 * a CUDA graph, and replay it with hesp_graph_launch (same buffers, current
 * contents).  Calls that synchronise (hesp_surrogate_fit_stats,
 * hesp_rank_metrics, hesp_sim_autotune, host copies) cannot be captured.
 * The first simulation call on a platform and device should come before a
 * capture (it sets the kernel's shared-memory attribute). */
typedef struct hesp_graph hesp_graph;
int hesp_graph_begin(void *stream);
int hesp_graph_end(void *stream, hesp_graph **out);
int hesp_graph_launch(const hesp_graph *g, void *stream);
void hesp_graph_destroy(hesp_graph *g);

/* Launch shape of the simulator for a platform: CTAs of 8 candidate warps per
 * SM (0 = as many as fit) and the place of the released-task bitmap (0 auto,
 * 1 global memory, 2 shared memory when it fits).  hesp_sim_autotune times a
 * sample batch (cands_dev, levels_dev, n_sample) under every shape, keeps the
 * fastest in `p` and appends it to cache_path (nullable); a cached entry for
 * the same GPU, bounds and platform shape is reused without timing.  ms_out
 * (nullable, [8]) receives the time of each shape (bitmap-major, -1 if not
 * run).  Synchronous; the workspace must hold the sample. */
int hesp_platform_set_tuning(hesp_platform *p, int32_t ctas_per_sm, int32_t bitmap_place);
int hesp_platform_get_tuning(const hesp_platform *p, int32_t *ctas_per_sm, int32_t *bitmap_place);
int hesp_sim_autotune(hesp_platform *p, const hesp_cand *cands_dev, const int8_t *levels_dev, int64_t n_sample,
                      int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t *makespan_dev,
                      int32_t *status_dev, void *workspace_dev, size_t workspace_bytes, const char *cache_path,
                      int32_t *best_ctas, int32_t *best_bitmap, float *ms_out, void *stream);

/* Largest-first ordering of a ragged batch (so that long simulations start
 * first and the batch ends together): sorted_dev[i] = cands_dev[perm_dev[i]]
 * in decreasing task count (buckets of 16 tasks; candidates in one bucket in
 * any order).  perm_dev nullable; workspace from
 * hesp_sort_cands_workspace_size. */
int hesp_sort_cands_workspace_size(int64_t n_cand, size_t *bytes_out);
int hesp_sort_cands_by_size(const hesp_cand *cands_dev, const int8_t *levels_dev, int64_t n_cand,
                            hesp_cand *sorted_dev, int32_t *perm_dev, void *workspace_dev, size_t workspace_bytes,
                            void *stream);

/* --------------------------------------------------- candidate generation
 * Partition vectors drawn on the device from SplitMix64 (Steele, Lea, Flood,
 * OOPSLA 2014) used as a counter-based generator: output k of candidate c is
 * mix(seed + ((c << 32) + k + 1) * 0x9E3779B97F4A7C15) and a draw in [0, m)
 * is ((u >> 32) * m) >> 32.  Candidates first .. first+n_cand-1 are written to
 * index 0 .. n_cand-1 (the search of Sec. 2.1 "Iterative solver" proposes
 * partitions; these are its random proposals). */
#define HESP_GEN_EXHAUSTIVE 0 /* level[c][t] = bit t of c (levels 0/1) */
#define HESP_GEN_UNIFORM 1    /* level[c][t] = draw(n_levels) at k = t */

/* Fixed (n_tiles, b): levels_dev[n_cand * n_base], cands_dev[n_cand]
 * (level_offset = c * n_base).  cands_dev may be NULL. */
int hesp_generate_candidates(int32_t kind, uint64_t seed, int64_t first, int64_t n_cand, int32_t n_tiles,
                             int32_t b, int32_t n_levels, hesp_cand *cands_dev, int8_t *levels_dev,
                             void *stream);

/* Local proposals around parents (the "repartition" moves of the partition
 * stage): proposal c copies parent (c mod n_parents) of parents_dev
 * [n_parents, n_base] and redraws each level with probability p_mut
 * (rounded to a multiple of 2^-16): the redraw test uses output k = 2t and
 * the new level draw(n_levels) output k = 2t + 1 of candidate first + c. */
int hesp_generate_mutants(const int8_t *parents_dev, int32_t n_parents, int32_t n_base, int32_t n_levels,
                          double p_mut, uint64_t seed, int64_t first, int64_t n, int8_t *levels_dev, void *stream);

/* Ragged batch: n = 4 + draw(29) at k = 0, b = {512, 1024, 2048}[draw(3)] at
 * k = 1, level of base task t from r = draw(10) at k = 2 + t mapped 0-4 -> 0,
 * 5-7 -> 1, 8-9 -> 2.  Writes cands_dev[n_cand] with prefix-summed
 * level_offset and the levels (capacity levels_cap bytes; ERR_CAPACITY
 * reported through *levels_used_dev = -1 when too small).  levels_used_dev
 * (device int64) receives the total. */
int hesp_generate_uneven(uint64_t seed, int64_t first, int64_t n_cand, hesp_cand *cands_dev, int8_t *levels_dev,
                         int64_t levels_cap, int64_t *levels_used_dev, void *stream);

/* ------------------------------------------------ tensor-core BF16 GEMM
 * The dense layers of the surrogate (below) run on this kernel; it is
 * exported for reuse and testing.  C[M, N] = A[M, K] . B[N, K]^T with A, B
 * bf16 row-major (leading dimensions lda, ldb >= K, multiples of 8 elements,
 * 16-byte aligned), K a multiple of 64, FP32 accumulation in tensor memory.
 * epilogue 0: c_dev[M, ldc] (fp32) = acc.
 * epilogue 1: out_dev[M, ldo] (bf16) = relu(acc + bias_dev[N]) (round to nearest even).
 * epilogue 2: out_dev[M, ldo] (bf16) = acc where mask_dev[M, ldm] (bf16) > 0, else 0.
 * out_t_dev (nullable, epilogues 1-2): the same values transposed, [N, ldt].
 * err_dev (nullable, device int32): set to 1 if a pipeline wait timed out. */
int hesp_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *a_dev, int64_t lda, const void *b_dev, int64_t ldb,
                   int32_t epilogue, float *c_dev, int64_t ldc, const float *bias_dev, void *out_dev, int64_t ldo,
                   void *out_t_dev, int64_t ldt, const void *mask_dev, int64_t ldm, int32_t *err_dev, void *stream);

/* ---------------------------------------------------------- surrogate MLP
 * Not in the paper: a learned model of the simulator that ranks proposals for
 * the partition stage of HeSP's search (Sec. 2.1 "Iterative solver"), so
 * that only the best-ranked ones are simulated exactly.
 * Input: the partition vector (n_base split levels in 0..n_levels-1), one-hot
 * encoded into F = n_base * n_levels features (padded with zeros to Fp, a
 * multiple of 64).  Network: F -> H -> H -> 1 with ReLU; bf16 weights and
 * activations (round to nearest even), FP32 accumulation on the tensor cores;
 * target t = (ln makespan - mu) / sigma; loss mean (y - t)^2; Adam
 * (beta 0.9 / 0.999, eps 1e-8) on FP32 masters.  Initial weights: He-uniform
 * from SplitMix64 (parameter id c = 0 for W1, 1 for W2, 2 for w3, element k
 * in row-major order: w = (2 f - 1) sqrt(6 / fan_in), f = (u >> 40) 2^-24),
 * biases 0.  The handle owns its device memory (weights, optimiser state and
 * activations for max_batch rows). */
typedef struct hesp_surrogate hesp_surrogate;

/* hidden and max_batch: multiples of 64; n_levels 1 .. HESP_MAX_LEVEL + 1
 * (the first layer builds its one-hot operand inside the GEMM from a table
 * sized for at most 5 levels).  Synchronous. */
int hesp_surrogate_create(int32_t n_base, int32_t n_levels, int32_t hidden, int32_t max_batch, uint64_t seed,
                          hesp_surrogate **out);
void hesp_surrogate_destroy(hesp_surrogate *s);
/* Checkpoints (synchronous, host files): hesp_surrogate_save writes the
 * shape, the seed, the Adam step count, the target standardisation (mu,
 * sigma), the FP32 parameters and both Adam moment tensors, followed by a
 * 64-bit FNV-1a hash of the file's bytes (written to path.tmp, then renamed).
 * hesp_surrogate_load creates a new handle from such a file: training resumed
 * from it continues exactly as the saved handle would.  ERR_ARG for a file
 * that cannot be written / read, has another layout, is truncated, carries
 * trailing bytes or fails the hash (then *out stays NULL). */
int hesp_surrogate_save(const hesp_surrogate *s, const char *path);
int hesp_surrogate_load(const char *path, hesp_surrogate **out);
int hesp_surrogate_shape(const hesp_surrogate *s, int64_t *F_out, int64_t *Fp_out, int32_t *H_out);
/* Target standardisation: set directly, or fit (mean and population standard
 * deviation of ln makespan over makespan_dev[n]; synchronises the stream). */
int hesp_surrogate_set_stats(hesp_surrogate *s, double mu, double sigma);
int hesp_surrogate_get_stats(const hesp_surrogate *s, double *mu, double *sigma, int64_t *adam_steps);
int hesp_surrogate_fit_stats(hesp_surrogate *s, const int64_t *makespan_dev, int64_t n, void *stream);
/* Host copies of the FP32 tensors in the order W1 [H, Fp], b1 [H], W2 [H, H],
 * b2 [H], w3 [H], b3 [1], n = total count; which: 0 parameters, 1 gradients,
 * 2 Adam first moments, 3 second moments (checkpoint / restore). Synchronous. */
int hesp_surrogate_get(const hesp_surrogate *s, int32_t which, float *host, int64_t n);
int hesp_surrogate_set(hesp_surrogate *s, int32_t which, const float *host, int64_t n);
/* Forward and backward on levels_dev [B, n_base] with makespan_dev [B]
 * (B a multiple of 64, <= max_batch): gradients into the handle; pred_dev [B]
 * and loss_dev [1] (fp32, nullable) receive y and the loss. */
int hesp_surrogate_grad(hesp_surrogate *s, const int8_t *levels_dev, const int64_t *makespan_dev, int32_t B,
                        float *pred_dev, float *loss_dev, void *stream);
/* One Adam update with the gradients held by the handle. */
int hesp_surrogate_adam(hesp_surrogate *s, float lr, void *stream);
/* n_steps updates on minibatches of `batch` rows drawn from n_samples
 * labelled samples (row i of step k = sample draw(u(seed, k, i), n_samples));
 * loss_dev [n_steps] (nullable) receives each step's loss. */
int hesp_surrogate_train(hesp_surrogate *s, const int8_t *levels_dev, const int64_t *makespan_dev, int64_t n_samples,
                         int32_t batch, int32_t n_steps, float lr, uint64_t seed, float *loss_dev, void *stream);
/* pred_dev[n] = predicted standardised log-makespan of levels_dev [n, n_base]
 * (processed in chunks of max_batch rows). */
int hesp_surrogate_infer(hesp_surrogate *s, const int8_t *levels_dev, int64_t n, float *pred_dev, void *stream);
/* 1 if a tensor-core pipeline wait of this handle timed out, else 0. */
int hesp_surrogate_error(hesp_surrogate *s, int32_t *err_host);

/* ------------------------------------------------- select and re-score
 * hesp_select_topk: indices (ascending) of the k smallest keys of keys_dev[n]
 * (ties broken by the lower index) into idx_dev[k]; workspace from
 * hesp_select_workspace_size (device, 16-byte aligned).
 * hesp_make_cands: cands_dev[k] = candidate (n_tiles, b) whose levels are row
 * idx_dev[i] of a [*, n_base] level array, for re-simulation.
 * hesp_gather_f32: dst_dev[i] = src_dev[idx_dev[i]].
 * hesp_rank_metrics: out_host[0] = mean |exp(pred sigma + mu) - makespan| /
 * makespan, out_host[1] = Spearman rank correlation (average ranks for ties)
 * of pred and makespan over k items; synchronises the stream. */
int hesp_select_workspace_size(int64_t n, size_t *bytes_out);
int hesp_select_topk(const float *keys_dev, int64_t n, int64_t k, int64_t *idx_dev, void *workspace_dev,
                     size_t workspace_bytes, void *stream);
int hesp_make_cands(const int64_t *idx_dev, int64_t k, int32_t n_tiles, int32_t b, hesp_cand *cands_dev,
                    void *stream);
int hesp_gather_f32(const float *src_dev, const int64_t *idx_dev, int64_t k, float *dst_dev, void *stream);
/* out_dev[0] = smallest makespan among candidates with status HESP_OK
 * (INT64_MAX if none), out_dev[1] = their total task count (ntasks_dev
 * nullable: 0). */
int hesp_best_makespan(const int64_t *makespan_dev, const int32_t *status_dev, const int64_t *ntasks_dev, int64_t n,
                       int64_t *out_dev, void *stream);
/* The best candidate of a batch, the result of one schedule stage over a
 * batch of partitions (Sec. 2.1 "Iterative solver": the partition with the
 * least simulated makespan is kept): out_dev[0] = the least makespan among
 * candidates with status HESP_OK (INT64_MAX if none), out_dev[1] =
 * first_index + the lowest index holding it (-1 if none).  first_index is
 * the global index of the batch's first candidate, so that the pairs of
 * several batches or ranks combine by taking the least (makespan, index).
 * out_dev: two int64 in device memory, written on `stream`. */
int hesp_best_candidate(const int64_t *makespan_dev, const int32_t *status_dev, int64_t n, int64_t first_index,
                        int64_t *out_dev, void *stream);
/* dst_dev[i, :] = src_dev[idx_dev[i], :] for int8 rows of `width` bytes. */
int hesp_gather_rows(const int8_t *src_dev, const int64_t *idx_dev, int64_t k, int64_t width, int8_t *dst_dev,
                     void *stream);
int hesp_rank_metrics_workspace_size(int64_t k, size_t *bytes_out);
int hesp_rank_metrics(const float *pred_dev, const int64_t *makespan_dev, int64_t k, double mu, double sigma,
                      void *workspace_dev, size_t workspace_bytes, double *out_host, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HESP_H */
