// Host side of the C ABI declared in include/hesp.h.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "hesp_internal.h"

namespace hesp {

int64_t tasks_uniform(int64_t n, int level) {
    const int64_t s = n << level;
    return s * (s + 1) * (s + 2) / 6;
}

int64_t regions_uniform(int64_t n, int level) {
    // tasks of the tiled algorithm on s = n 2^level tiles, weighted by their
    // region count (chol 1, trsm 2, syrk 2, gemm 3)
    const int64_t s = n << level;
    const int64_t trsm = s * (s - 1) / 2, syrk = trsm, gemm = s * (s - 1) * (s - 2) / 6;
    return s + 2 * trsm + 2 * syrk + 3 * gemm;
}

static int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

Arena arena_offsets(Arena a, int32_t n_mem, unsigned room);

unsigned arena_room_of(const hesp_platform *p) {
    return (p->order == HESP_ORDER_PL ? kRoomPL : 0u) | (p->use_cap ? kRoomCap : 0u);
}

Arena make_arena(int32_t max_tiles, int32_t max_level, int32_t n_mem, int64_t task_cap, unsigned room) {
    Arena a;
    memset(&a, 0, sizeof a);
    const int64_t tb = tasks_uniform(max_tiles, max_level), eb = regions_uniform(max_tiles, max_level);
    // without a cap the closed-form bounds hold every candidate; with one,
    // larger candidates are reported as HESP_ERR_CAPACITY
    a.Tcap = task_cap > 0 && task_cap < tb ? task_cap : tb;
    a.Ecap = task_cap > 0 && 4 * a.Tcap < eb ? 4 * a.Tcap : eb;
    a.Acap = ((int64_t)max_tiles * (max_tiles + 1) / 2) << (2 * max_level);
    a.Kcap = (3LL << (2 * max_level)) + 1;
    return arena_offsets(a, n_mem, room);
}

// Offsets of the arena areas for the capacities in a.  The link area holds,
// one after the other in time, the edge list of the dependence build (4
// bytes per edge), the FIFO records of the event loop (16 bytes per task),
// or the four per-task words of the priority-list order (32 bytes per task,
// only with kRoomPL) and the two of the critical-path pass (16).
Arena arena_offsets(Arena a, int32_t n_mem, unsigned room) {
    const int64_t mp = n_mem <= 1 ? 0 : (n_mem == 2 ? 2 : 4);  // int64 words of coherence state per atom
    const int64_t per_task = (room & kRoomPL) ? 32 : 16;
    const int64_t link_bytes = per_task * a.Tcap > 4 * a.Ecap ? per_task * a.Tcap : 4 * a.Ecap;
    int64_t o = 0;
    a.off_desc = o; o = align256(o + 8 * a.Tcap);
    a.off_pending = o; o = align256(o + 2 * a.Tcap);
    a.off_link = o; o = align256(o + link_bytes);
    a.off_epred = a.off_link;
    a.off_next = o; o = align256(o + 4 * a.Tcap);
    a.off_succoff = o; o = align256(o + 4 * (a.Tcap + 1));
    a.off_succ = o; o = align256(o + 4 * a.Ecap);
    a.off_lw = o; o = align256(o + 4 * a.Acap);
    a.off_vfrom = o; o = align256(o + 8 * a.Acap * mp);
    a.off_bitmap = o; o = align256(o + 4 * ((a.Tcap + 31) / 32));
    a.off_xt = o; o = align256(o + 8 * a.Kcap * (n_mem > 1 ? HESP_MAX_MEMS * HESP_MAX_MEMS : 1));  // per link
    a.off_hist = o; o = align256(o + 4 * 256);  // radix histogram of the priority-list sort
    // keep / reuse: the DAG's initial pending counts and the candidate's header
    a.off_pend0 = o; o = align256(o + ((room & kRoomKept) ? 2 * a.Tcap : 0));
    a.off_hdr = o; o = align256(o + ((room & kRoomKept) ? 64 : 0));
    // finite memories: last use per atom and memory
    a.off_use = o; o = align256(o + ((room & kRoomCap) ? 8 * a.Acap * mp : 0));
    a.slot_bytes = o;
    return a;
}

// Least common multiple of 1 .. max_factor: atoms per tile side in factor mode.
int32_t factor_lcm(int32_t max_factor) {
    int32_t L = 1;
    for (int32_t f = 2; f <= max_factor; ++f) {
        int32_t x = L, y = f;
        while (y) {
            const int32_t r = x % y;
            x = y;
            y = r;
        }
        L = L / x * f;
    }
    return L;
}

// Arena of one-level k-way partitions with factors up to max_factor: the
// tasks of every base task cut max_factor ways, atoms of side b / lcm(1 ..
// max_factor), edges up to 16 per task (a larger DAG reports
// HESP_ERR_CAPACITY).
Arena make_arena_factors(int32_t max_tiles, int32_t max_factor, int32_t n_mem, int64_t task_cap, unsigned room) {
    Arena a;
    memset(&a, 0, sizeof a);
    const int64_t n = max_tiles, k = max_factor;
    const int64_t tb = n * (k * (k + 1) * (k + 2) / 6) + n * (n - 1) * (k * k * (k + 1) / 2) +
                       n * (n - 1) * (n - 2) / 6 * (k * k * k);
    a.Tcap = task_cap > 0 && task_cap < tb ? task_cap : tb;
    a.Ecap = 16 * a.Tcap;
    const int64_t L = factor_lcm(max_factor);
    a.Acap = n * (n + 1) / 2 * L * L;
    a.Kcap = 3 * L * L + 1;
    return arena_offsets(a, n_mem, room);
}

static DevPlatform dev_platform(const hesp_platform *p) {
    DevPlatform d;
    memset(&d, 0, sizeof d);
    d.n_mem = p->n_mem;
    d.n_types = p->n_types;
    d.n_procs = p->n_procs;
    for (int op = 0; op < 4; ++op)
        for (int t = 0; t < HESP_MAX_TYPES; ++t)
            for (int l = 0; l < HESP_LB; ++l) d.exec[(op * HESP_MAX_TYPES + t) * HESP_LB + l] = p->exec[op][t][l];
    for (int i = 0; i < p->n_procs; ++i) {
        d.proc_mem[i] = (int8_t)p->procs[i].memory;
        d.proc_type[i] = (int8_t)p->procs[i].type;
    }
    d.order = p->order;
    d.select = p->select;
    d.rp_seed = p->rp_seed;
    d.cache = p->cache;
    d.use_links = p->use_links;
    d.use_cap = p->use_cap;
    for (int m = 0; m < HESP_MAX_MEMS; ++m) d.cap_bytes[m] = p->cap_bytes[m];
    for (int s = 0; s < HESP_MAX_MEMS; ++s)
        for (int t = 0; t < HESP_MAX_MEMS; ++t) {
            d.link_lat[s * HESP_MAX_MEMS + t] = p->use_links ? p->link_lat[s][t] : p->xfer_latency_ns;
            d.link_bw[s * HESP_MAX_MEMS + t] = p->use_links ? p->link_bw[s][t] : p->bw_bytes_per_ns;
        }
    for (int op = 0; op < 4; ++op)
        for (int l = 0; l < HESP_LB; ++l) {
            int64_t s = 0;
            for (int i = 0; i < p->n_procs && s >= 0; ++i) {
                const int64_t e = p->exec[op][p->procs[i].type][l];
                s = (e < 0 || s + e >= (1LL << 40)) ? -1 : s + e;
            }
            d.wsum[op * HESP_LB + l] = s;
        }
    d.lat = p->xfer_latency_ns;
    d.bpe = p->bytes_per_elem;
    d.bw = p->bw_bytes_per_ns;
    return d;
}

// Task time of (op, type) on a bs x bs block: ceil(flops / rate) with
// flops = c bs^3 / 3 and rate = peak eff/100 bs^2 / (bs^2 + h^2), i.e.
// ceil(c bs (bs^2 + h^2) 100 / (3 peak eff)); -1 if above 2^56.
static int64_t model_exec(const hesp_ptype &ty, int op, int64_t bs) {
    static const int64_t coef[4] = {1, 3, 3, 6};
    const unsigned __int128 num =
        (unsigned __int128)coef[op] * (unsigned __int128)bs * ((unsigned __int128)bs * bs + (unsigned __int128)ty.h * ty.h) * 100u;
    const unsigned __int128 den = (unsigned __int128)3 * (unsigned __int128)ty.peak_gflops * (unsigned __int128)ty.eff_pct[op];
    const unsigned __int128 q = (num + den - 1) / den;
    if (q >= ((unsigned __int128)1 << 56)) return -1;
    return (int64_t)q;
}


// Factor mode: exec and wsum indexed by the factor k (1 .. max_factor) for
// blocks of b / k: the platform's table where b / k is a power of two (so
// that measured-model overrides apply), else the performance model; -1
// where b / k is not an integer.
static DevPlatform dev_platform_factors(const hesp_platform *p, int32_t b, int32_t max_factor) {
    DevPlatform d = dev_platform(p);
    for (int op = 0; op < 4; ++op) {
        for (int t = 0; t < HESP_MAX_TYPES; ++t)
            for (int k = 1; k <= max_factor; ++k) {
                int64_t e = -1;
                if (t < p->n_types && b % k == 0) {
                    const int64_t bs = b / k;
                    int l = 0;
                    while ((1LL << l) < bs) ++l;
                    e = (1LL << l) == bs && l < HESP_LB ? p->exec[op][t][l] : model_exec(p->types[t], op, bs);
                }
                d.exec[(op * HESP_MAX_TYPES + t) * HESP_LB + k] = e;
            }
        for (int k = 1; k <= max_factor; ++k) {
            int64_t s = 0;
            for (int i = 0; i < p->n_procs && s >= 0; ++i) {
                const int64_t e = d.exec[(op * HESP_MAX_TYPES + p->procs[i].type) * HESP_LB + k];
                s = (e < 0 || s + e >= (1LL << 40)) ? -1 : s + e;
            }
            d.wsum[op * HESP_LB + k] = s;
        }
    }
    return d;
}

// Resident warps of the simulation kernel on the current device.
int sim_slots_for(const hesp_platform *p, const Arena &ar, int64_t *resident_warps) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HESP_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HESP_ERR_CUDA;
    int blocks = 0, threads = 0;
    int rc = sim_kernel_occupancy(p->n_mem, p->n_procs, ar.Tcap, &blocks, &threads);
    if (rc) return rc;
    if (blocks < 1) blocks = 1;
    // the tuning value counts groups of 8 candidate warps per SM
    const int per8 = threads >= 256 ? 1 : 256 / threads;
    if (p->tune_ctas_per_sm > 0 && p->tune_ctas_per_sm * per8 < blocks) blocks = p->tune_ctas_per_sm * per8;
    *resident_warps = (int64_t)sms * blocks * (threads / 32);
    return HESP_OK;
}

}  // namespace hesp

using namespace hesp;

extern "C" {

const char *hesp_status_string(int s) {
    switch (s) {
    case HESP_OK: return "HESP_OK";
    case HESP_ERR_ARG: return "HESP_ERR_ARG";
    case HESP_ERR_CAPACITY: return "HESP_ERR_CAPACITY";
    case HESP_ERR_CUDA: return "HESP_ERR_CUDA";
    case HESP_ERR_TIMEOUT: return "HESP_ERR_TIMEOUT";
    case HESP_ERR_STATE: return "HESP_ERR_STATE";
    case HESP_ERR_UNSUPPORTED: return "HESP_ERR_UNSUPPORTED";
    default: return "HESP_ERR_UNKNOWN";
    }
}

int hesp_platform_create(const hesp_platform_desc *d, hesp_platform **out) {
    if (!d || !out) return HESP_ERR_ARG;
    *out = nullptr;
    if (d->n_mem < 1 || d->n_types < 1 || d->n_procs < 1 || !d->types || !d->procs) return HESP_ERR_ARG;
    if (d->n_mem > HESP_MAX_MEMS || d->n_types > HESP_MAX_TYPES || d->n_procs > HESP_MAX_PROCS)
        return HESP_ERR_UNSUPPORTED;
    if (d->xfer_latency_ns < 0 || d->bytes_per_elem < 1 || (d->n_mem > 1 && d->bw_bytes_per_ns < 1))
        return HESP_ERR_ARG;
    if (d->xfer_latency_ns > (1LL << 40) || d->bytes_per_elem > (1 << 20)) return HESP_ERR_UNSUPPORTED;
    for (int t = 0; t < d->n_types; ++t) {
        const hesp_ptype &ty = d->types[t];
        if (ty.peak_gflops < 1 || ty.h < 0 || ty.peak_gflops > (1LL << 40) || ty.h > (1LL << 30)) return HESP_ERR_ARG;
        for (int o = 0; o < 4; ++o)
            if (ty.eff_pct[o] < 1 || ty.eff_pct[o] > 100000) return HESP_ERR_ARG;
    }
    for (int i = 0; i < d->n_procs; ++i)
        if (d->procs[i].memory < 0 || d->procs[i].memory >= d->n_mem || d->procs[i].type < 0 ||
            d->procs[i].type >= d->n_types)
            return HESP_ERR_ARG;
    hesp_platform *p = (hesp_platform *)calloc(1, sizeof(hesp_platform));
    if (!p) return HESP_ERR_CAPACITY;
    p->n_mem = d->n_mem;
    p->n_types = d->n_types;
    p->n_procs = d->n_procs;
    p->xfer_latency_ns = d->xfer_latency_ns;
    p->bytes_per_elem = d->bytes_per_elem;
    p->bw_bytes_per_ns = d->n_mem > 1 ? d->bw_bytes_per_ns : (d->bw_bytes_per_ns > 0 ? d->bw_bytes_per_ns : 1);
    memcpy(p->types, d->types, sizeof(hesp_ptype) * d->n_types);
    memcpy(p->procs, d->procs, sizeof(hesp_proc) * d->n_procs);
    for (int op = 0; op < 4; ++op)
        for (int t = 0; t < HESP_MAX_TYPES; ++t)
            for (int l = 0; l < HESP_LB; ++l)
                p->exec[op][t][l] = t < d->n_types ? model_exec(p->types[t], op, (int64_t)1 << l) : -1;
    *out = p;
    return HESP_OK;
}

static int log2_exact(int64_t v) {
    if (v < 1 || (v & (v - 1))) return -1;
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
}

int hesp_platform_set_exec_table(hesp_platform *p, int32_t op, int32_t type, int64_t block, int64_t ns) {
    if (!p || op < 0 || op > 3 || type < 0 || type >= p->n_types || ns < 1 || ns >= (1LL << 56)) return HESP_ERR_ARG;
    const int l = log2_exact(block);
    if (l < 0 || l > HESP_MAX_LOG2_BLOCK) return HESP_ERR_ARG;
    p->exec[op][type][l] = ns;
    return HESP_OK;
}

int hesp_platform_set_policy(hesp_platform *p, int32_t order, int32_t select, uint64_t rp_seed) {
    if (!p || order < HESP_ORDER_FCFS || order > HESP_ORDER_PL || select < HESP_SELECT_EFT ||
        select > HESP_SELECT_RP)
        return HESP_ERR_ARG;
    p->order = order;
    p->select = select;
    p->rp_seed = rp_seed;
    return HESP_OK;
}

int hesp_platform_set_link(hesp_platform *p, int32_t src, int32_t dst, int64_t latency_ns, int64_t bw_bytes_per_ns) {
    if (!p || src < 0 || dst < 0 || src >= p->n_mem || dst >= p->n_mem || src == dst || latency_ns < 0 ||
        bw_bytes_per_ns < 1)
        return HESP_ERR_ARG;
    if (latency_ns > (1LL << 40)) return HESP_ERR_UNSUPPORTED;
    if (!p->use_links) {  // every other pair keeps the platform's scalars
        for (int s = 0; s < HESP_MAX_MEMS; ++s)
            for (int t = 0; t < HESP_MAX_MEMS; ++t) {
                p->link_lat[s][t] = p->xfer_latency_ns;
                p->link_bw[s][t] = p->bw_bytes_per_ns;
            }
        p->use_links = 1;
    }
    p->link_lat[src][dst] = latency_ns;
    p->link_bw[src][dst] = bw_bytes_per_ns;
    return HESP_OK;
}

int hesp_platform_set_capacity(hesp_platform *p, int32_t mem, int64_t bytes) {
    if (!p || mem < 1 || mem >= p->n_mem || bytes < 0) return HESP_ERR_ARG;
    p->cap_bytes[mem] = bytes;
    p->use_cap = 0;
    for (int m = 1; m < p->n_mem; ++m)
        if (p->cap_bytes[m] > 0) p->use_cap = 1;
    return HESP_OK;
}

int hesp_platform_set_cache(hesp_platform *p, int32_t cache) {
    if (!p || cache < HESP_CACHE_WB || cache > HESP_CACHE_WA) return HESP_ERR_ARG;
    p->cache = cache;
    return HESP_OK;
}

int hesp_platform_exec_ns(const hesp_platform *p, int32_t op, int32_t type, int64_t block, int64_t *ns_out) {
    if (!p || !ns_out || op < 0 || op > 3 || type < 0 || type >= p->n_types) return HESP_ERR_ARG;
    const int l = log2_exact(block);
    if (l < 0 || l > HESP_MAX_LOG2_BLOCK) return HESP_ERR_ARG;
    if (p->exec[op][type][l] < 0) return HESP_ERR_UNSUPPORTED;
    *ns_out = p->exec[op][type][l];
    return HESP_OK;
}

int hesp_platform_xfer_ns(const hesp_platform *p, int64_t elems, int64_t *ns_out) {
    if (!p || !ns_out || elems < 0) return HESP_ERR_ARG;
    const unsigned __int128 bytes = (unsigned __int128)elems * (unsigned __int128)p->bytes_per_elem;
    const unsigned __int128 q = (bytes + p->bw_bytes_per_ns - 1) / (unsigned __int128)p->bw_bytes_per_ns;
    if (q >= ((unsigned __int128)1 << 60)) return HESP_ERR_UNSUPPORTED;
    *ns_out = p->xfer_latency_ns + (int64_t)q;
    return HESP_OK;
}

void hesp_platform_destroy(hesp_platform *p) { free(p); }

// ------------------------------------------------------------------- DAG

int hesp_dag_build(int32_t n_tiles, int32_t b, int32_t max_level, hesp_dag **out) {
    if (!out) return HESP_ERR_ARG;
    *out = nullptr;
    if (n_tiles < 1 || max_level < 0 || b < 1) return HESP_ERR_ARG;
    if (n_tiles > HESP_MAX_TILES || max_level > HESP_MAX_LEVEL || log2_exact(b) < 0 ||
        log2_exact(b) > HESP_MAX_LOG2_BLOCK || (b >> max_level) < 1)
        return HESP_ERR_UNSUPPORTED;
    hesp_dag *d = (hesp_dag *)calloc(1, sizeof(hesp_dag));
    if (!d) return HESP_ERR_CAPACITY;
    d->n_tiles = n_tiles;
    d->b = b;
    d->max_level = max_level;
    d->n_base = (int64_t)n_tiles * (n_tiles + 1) * (n_tiles + 2) / 6;
    d->op = (int32_t *)malloc(sizeof(int32_t) * d->n_base);
    d->k = (int32_t *)malloc(sizeof(int32_t) * d->n_base);
    d->i = (int32_t *)malloc(sizeof(int32_t) * d->n_base);
    d->j = (int32_t *)malloc(sizeof(int32_t) * d->n_base);
    if (!d->op || !d->k || !d->i || !d->j) {
        hesp_dag_destroy(d);
        return HESP_ERR_CAPACITY;
    }
    int64_t t = 0;
    for (int k = 0; k < n_tiles; ++k) {
        d->op[t] = HESP_OP_CHOL; d->k[t] = k; d->i[t] = k; d->j[t] = k; ++t;
        for (int j = k + 1; j < n_tiles; ++j) { d->op[t] = HESP_OP_TRSM; d->k[t] = k; d->i[t] = k; d->j[t] = j; ++t; }
        for (int i = k + 1; i < n_tiles; ++i) {
            for (int j = i + 1; j < n_tiles; ++j) { d->op[t] = HESP_OP_GEMM; d->k[t] = k; d->i[t] = i; d->j[t] = j; ++t; }
            d->op[t] = HESP_OP_SYRK; d->k[t] = k; d->i[t] = i; d->j[t] = i; ++t;
        }
    }
    *out = d;
    return HESP_OK;
}

int64_t hesp_dag_n_base(const hesp_dag *d) { return d ? d->n_base : HESP_ERR_ARG; }

int hesp_dag_base_tasks(const hesp_dag *d, int32_t *op, int32_t *k, int32_t *i, int32_t *j) {
    if (!d || !op || !k || !i || !j) return HESP_ERR_ARG;
    memcpy(op, d->op, sizeof(int32_t) * d->n_base);
    memcpy(k, d->k, sizeof(int32_t) * d->n_base);
    memcpy(i, d->i, sizeof(int32_t) * d->n_base);
    memcpy(j, d->j, sizeof(int32_t) * d->n_base);
    return HESP_OK;
}

// Number of tasks of each op produced by an op split l times (2x2 blocked
// algorithms: chol -> chol, trsm, syrk, chol; trsm -> 4 trsm, 2 gemm;
// syrk -> 2 gemm, 4 syrk; gemm -> 8 gemm).
static void split_op_counts(int64_t tab[4][HESP_MAX_LEVEL + 1][4]) {
    static const int kids[4][4] = {{2, 1, 1, 0}, {0, 4, 0, 2}, {0, 0, 4, 2}, {0, 0, 0, 8}};  // [op][child op]
    for (int op = 0; op < 4; ++op)
        for (int o = 0; o < 4; ++o) tab[op][0][o] = op == o;
    for (int l = 1; l <= HESP_MAX_LEVEL; ++l)
        for (int op = 0; op < 4; ++op)
            for (int o = 0; o < 4; ++o) {
                int64_t v = 0;
                for (int c = 0; c < 4; ++c) v += kids[op][c] * tab[c][l - 1][o];
                tab[op][l][o] = v;
            }
}

int hesp_dag_count_tasks(const hesp_dag *d, const int8_t *levels, int64_t *n_tasks, int64_t *flops3) {
    if (!d || !levels || !n_tasks) return HESP_ERR_ARG;
    int64_t tab[4][HESP_MAX_LEVEL + 1][4];
    split_op_counts(tab);
    static const int64_t coef[4] = {1, 3, 3, 6};
    int64_t tot = 0;
    unsigned __int128 f = 0;
    for (int64_t t = 0; t < d->n_base; ++t) {
        const int l = levels[t];
        if (l < 0 || l > d->max_level) return HESP_ERR_ARG;
        const unsigned __int128 bs = (unsigned __int128)(d->b >> l);
        for (int o = 0; o < 4; ++o) {
            tot += tab[d->op[t]][l][o];
            f += (unsigned __int128)tab[d->op[t]][l][o] * coef[o] * bs * bs * bs;
        }
    }
    *n_tasks = tot;
    if (flops3) *flops3 = (int64_t)f;
    return HESP_OK;
}

void hesp_dag_destroy(hesp_dag *d) {
    if (!d) return;
    free(d->op);
    free(d->k);
    free(d->i);
    free(d->j);
    free(d);
}

// ---------------------------------------------------------- simulation

int hesp_sim_workspace_size(const hesp_platform *p, int32_t max_tiles, int32_t max_level, int64_t task_cap,
                            int64_t n_cand, size_t *bytes_out) {
    if (!p || !bytes_out || n_cand < 0 || task_cap < 0) return HESP_ERR_ARG;
    if (max_tiles < 1 || max_tiles > HESP_MAX_TILES || max_level < 0 || max_level > HESP_MAX_LEVEL)
        return HESP_ERR_UNSUPPORTED;
    const Arena ar = make_arena(max_tiles, max_level, p->n_mem, task_cap, arena_room_of(p));
    int64_t resident = 0;
    const int rc = sim_slots_for(p, ar, &resident);
    if (rc) return rc;
    int64_t slots = n_cand < resident ? n_cand : resident;
    if (slots < 1) slots = 1;
    *bytes_out = (size_t)(kWsHeaderBytes + slots * ar.slot_bytes);
    return HESP_OK;
}

namespace {

int simulate_common(const hesp_platform *p, const hesp_cand *cands, const int8_t *levels, int64_t n_cand,
                    int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t *makespan, int32_t *status,
                    int64_t *ntasks, const int64_t *sched_off, int16_t *sproc, int64_t *sstart, int64_t *sfinish,
                    int8_t *crit, void *ws, size_t ws_bytes, void *stream) {
    if (!p || n_cand < 0 || task_cap < 0) return HESP_ERR_ARG;
    if (n_cand == 0) return HESP_OK;
    if (!cands || !levels || !makespan || !status || !ws) return HESP_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return HESP_ERR_ARG;
    const bool any_s = sched_off || sproc || sstart || sfinish;
    const bool all_s = sched_off && sproc && sstart && sfinish;
    if (any_s && !all_s) return HESP_ERR_ARG;
    if (max_tiles < 1 || max_tiles > HESP_MAX_TILES || max_level < 0 || max_level > HESP_MAX_LEVEL)
        return HESP_ERR_UNSUPPORTED;
    if (p->use_cap && p->select >= HESP_SELECT_FP) return HESP_ERR_ARG;  // finite memories: EFT-P / EIT-P
    const Arena ar = make_arena(max_tiles, max_level, p->n_mem, task_cap, arena_room_of(p));
    if ((int64_t)ws_bytes < kWsHeaderBytes + ar.slot_bytes) return HESP_ERR_ARG;
    int64_t resident = 0;
    int rc = sim_slots_for(p, ar, &resident);
    if (rc) return rc;
    int64_t slots = ((int64_t)ws_bytes - kWsHeaderBytes) / ar.slot_bytes;
    if (slots > resident) slots = resident;
    if (slots > n_cand) slots = n_cand;
    const DevPlatform dp = dev_platform(p);
    return launch_sim(p, dp, ar, slots, cands, levels, n_cand, max_tiles, max_level, makespan, status, ntasks,
                      sched_off, sproc, sstart, sfinish, crit, 0, 0, 0, 0, (char *)ws, (cudaStream_t)stream);
}

// Layout signature of keep / reuse arenas: their layout fields, mixed.
uint64_t layout_signature(const Arena &ar, int32_t max_tiles, int32_t max_level) {
    const uint64_t f[8] = {(uint64_t)ar.slot_bytes, (uint64_t)ar.Tcap, (uint64_t)ar.Ecap, (uint64_t)ar.Acap,
                           (uint64_t)ar.off_pend0, (uint64_t)ar.off_hdr, (uint64_t)max_tiles, (uint64_t)max_level};
    uint64_t h = 0x8C6B0F2D1E3A5947ull;
    for (int i = 0; i < 8; ++i) {
        h ^= f[i] + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    }
    return h | 1;  // never 0, so a zeroed arena never matches
}

// Keep (dag_mode 1) and reuse (dag_mode 2): one arena per candidate, laid
// out for the largest memory count so every platform uses the same offsets.
int simulate_kept(const hesp_platform *p, const hesp_cand *cands, const int8_t *levels, int64_t n_cand,
                  int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t *makespan, int32_t *status,
                  int64_t *ntasks, int dag_mode, void *ws, size_t ws_bytes, void *stream) {
    if (!p || n_cand < 0 || task_cap < 0) return HESP_ERR_ARG;
    if (n_cand == 0) return HESP_OK;
    if (!cands || !levels || !makespan || !status || !ws) return HESP_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return HESP_ERR_ARG;
    if (max_tiles < 1 || max_tiles > HESP_MAX_TILES || max_level < 0 || max_level > HESP_MAX_LEVEL)
        return HESP_ERR_UNSUPPORTED;
    if (p->use_cap && p->select >= HESP_SELECT_FP) return HESP_ERR_ARG;  // finite memories: EFT-P / EIT-P
    const Arena ar = make_arena(max_tiles, max_level, HESP_MAX_MEMS, task_cap, kRoomAll);
    if ((int64_t)ws_bytes < kWsHeaderBytes || ((int64_t)ws_bytes - kWsHeaderBytes) / ar.slot_bytes < n_cand)
        return HESP_ERR_ARG;
    int64_t resident = 0;
    int rc = sim_slots_for(p, ar, &resident);
    if (rc) return rc;
    const int64_t warps = resident < n_cand ? resident : n_cand;
    const DevPlatform dp = dev_platform(p);
    return launch_sim(p, dp, ar, warps, cands, levels, n_cand, max_tiles, max_level, makespan, status, ntasks,
                      nullptr, nullptr, nullptr, nullptr, nullptr, dag_mode, layout_signature(ar, max_tiles, max_level),
                      0, 0, (char *)ws, (cudaStream_t)stream);
}

}  // namespace

int hesp_simulate_batch(const hesp_platform *p, const hesp_cand *cands, const int8_t *levels, int64_t n_cand,
                        int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t *makespan, int32_t *status,
                        int64_t *ntasks,
                        const int64_t *sched_off, int16_t *sproc, int64_t *sstart, int64_t *sfinish, void *ws,
                        size_t ws_bytes, void *stream) {
    return simulate_common(p, cands, levels, n_cand, max_tiles, max_level, task_cap, makespan, status, ntasks,
                           sched_off, sproc, sstart, sfinish, nullptr, ws, ws_bytes, stream);
}

int hesp_sim_workspace_size_factors(const hesp_platform *p, int32_t max_tiles, int32_t max_factor, int64_t task_cap,
                                    int64_t n_cand, size_t *bytes_out) {
    if (!p || !bytes_out || n_cand < 0 || task_cap < 0) return HESP_ERR_ARG;
    if (max_tiles < 1 || max_tiles > HESP_MAX_TILES || max_factor < 1 || max_factor > HESP_MAX_FACTOR)
        return HESP_ERR_UNSUPPORTED;
    const Arena ar = make_arena_factors(max_tiles, max_factor, p->n_mem, task_cap, arena_room_of(p));
    int64_t resident = 0;
    const int rc = sim_slots_for(p, ar, &resident);
    if (rc) return rc;
    int64_t slots = n_cand < resident ? n_cand : resident;
    if (slots < 1) slots = 1;
    *bytes_out = (size_t)(kWsHeaderBytes + slots * ar.slot_bytes);
    return HESP_OK;
}

int hesp_simulate_factors(const hesp_platform *p, const hesp_cand *cands, const int8_t *factors, int64_t n_cand,
                          int32_t max_tiles, int32_t max_factor, int32_t b, int64_t task_cap, int64_t *makespan,
                          int32_t *status, int64_t *ntasks, const int64_t *sched_off, int16_t *sproc, int64_t *sstart,
                          int64_t *sfinish, int8_t *crit, void *ws, size_t ws_bytes, void *stream) {
    if (!p || n_cand < 0 || task_cap < 0) return HESP_ERR_ARG;
    if (n_cand == 0) return HESP_OK;
    if (!cands || !factors || !makespan || !status || !ws || b < 1) return HESP_ERR_ARG;
    if (p->use_cap) return HESP_ERR_UNSUPPORTED;  // finite memories: dyadic partitions only
    if (((uintptr_t)ws & 255) != 0) return HESP_ERR_ARG;
    const bool any_s = sched_off || sproc || sstart || sfinish;
    const bool all_s = sched_off && sproc && sstart && sfinish;
    if (any_s && !all_s) return HESP_ERR_ARG;
    if (max_tiles < 1 || max_tiles > HESP_MAX_TILES || max_factor < 1 || max_factor > HESP_MAX_FACTOR ||
        b > (1 << HESP_MAX_LOG2_BLOCK))
        return HESP_ERR_UNSUPPORTED;
    const Arena ar = make_arena_factors(max_tiles, max_factor, p->n_mem, task_cap, arena_room_of(p));
    if ((int64_t)ws_bytes < kWsHeaderBytes + ar.slot_bytes) return HESP_ERR_ARG;
    int64_t resident = 0;
    int rc = sim_slots_for(p, ar, &resident);
    if (rc) return rc;
    int64_t slots = ((int64_t)ws_bytes - kWsHeaderBytes) / ar.slot_bytes;
    if (slots > resident) slots = resident;
    if (slots > n_cand) slots = n_cand;
    const DevPlatform dp = dev_platform_factors(p, b, max_factor);
    return launch_sim(p, dp, ar, slots, cands, factors, n_cand, max_tiles, max_factor, makespan, status, ntasks,
                      sched_off, sproc, sstart, sfinish, crit, 0, 0, 1, b, (char *)ws, (cudaStream_t)stream);
}

int hesp_schedule_metrics(const hesp_cand *cands, const int8_t *levels, int64_t n_cand, const int64_t *sched_off,
                          const int64_t *start, const int64_t *finish, int64_t *busy, int64_t *ntasks,
                          int64_t *sum_block, int32_t *depth, void *stream) {
    if (n_cand < 0) return HESP_ERR_ARG;
    if (n_cand == 0) return HESP_OK;
    if (!cands || !levels) return HESP_ERR_ARG;
    const bool any_s = sched_off || start || finish;
    if (any_s && !(sched_off && start && finish)) return HESP_ERR_ARG;
    return launch_metrics(cands, levels, n_cand, sched_off, start, finish, busy, ntasks, sum_block, depth,
                          (cudaStream_t)stream);
}

int hesp_sim_workspace_size_kept(int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t n_cand,
                                 size_t *bytes_out) {
    if (!bytes_out || n_cand < 0 || task_cap < 0) return HESP_ERR_ARG;
    if (max_tiles < 1 || max_tiles > HESP_MAX_TILES || max_level < 0 || max_level > HESP_MAX_LEVEL)
        return HESP_ERR_UNSUPPORTED;
    const Arena ar = make_arena(max_tiles, max_level, HESP_MAX_MEMS, task_cap, kRoomAll);
    *bytes_out = (size_t)(kWsHeaderBytes + n_cand * ar.slot_bytes);
    return HESP_OK;
}

int hesp_dag_build_kept(const hesp_cand *cands, const int8_t *levels, int64_t n_cand, int32_t max_tiles,
                        int32_t max_level, int64_t task_cap, int32_t *status, int64_t *ntasks, void *ws,
                        size_t ws_bytes, void *stream) {
    if (n_cand < 0 || task_cap < 0) return HESP_ERR_ARG;
    if (n_cand == 0) return HESP_OK;
    if (!cands || !levels || !status || !ws || ((uintptr_t)ws & 255) != 0) return HESP_ERR_ARG;
    if (max_tiles < 1 || max_tiles > HESP_MAX_TILES || max_level < 0 || max_level > HESP_MAX_LEVEL)
        return HESP_ERR_UNSUPPORTED;
    const Arena ar = make_arena(max_tiles, max_level, HESP_MAX_MEMS, task_cap, kRoomAll);
    if ((int64_t)ws_bytes < kWsHeaderBytes || ((int64_t)ws_bytes - kWsHeaderBytes) / ar.slot_bytes < n_cand)
        return HESP_ERR_ARG;
    return launch_build(ar, cands, levels, n_cand, max_tiles, max_level, ntasks, status,
                        layout_signature(ar, max_tiles, max_level), (char *)ws, (cudaStream_t)stream);
}

int hesp_simulate_batch_keep(const hesp_platform *p, const hesp_cand *cands, const int8_t *levels, int64_t n_cand,
                             int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t *makespan,
                             int32_t *status, int64_t *ntasks, void *ws, size_t ws_bytes, void *stream) {
    return simulate_kept(p, cands, levels, n_cand, max_tiles, max_level, task_cap, makespan, status, ntasks, 1, ws,
                         ws_bytes, stream);
}

int hesp_simulate_batch_reuse(const hesp_platform *p, const hesp_cand *cands, const int8_t *levels, int64_t n_cand,
                              int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t *makespan,
                              int32_t *status, int64_t *ntasks, void *ws, size_t ws_bytes, void *stream) {
    return simulate_kept(p, cands, levels, n_cand, max_tiles, max_level, task_cap, makespan, status, ntasks, 2, ws,
                         ws_bytes, stream);
}

int hesp_simulate_critical(const hesp_platform *p, const hesp_cand *cands, const int8_t *levels, int64_t n_cand,
                           int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t *makespan,
                           int32_t *status, int8_t *crit, void *ws, size_t ws_bytes, void *stream) {
    if (n_cand > 0 && !crit) return HESP_ERR_ARG;
    return simulate_common(p, cands, levels, n_cand, max_tiles, max_level, task_cap, makespan, status, nullptr,
                           nullptr, nullptr, nullptr, nullptr, crit, ws, ws_bytes, stream);
}

int hesp_generate_candidates(int32_t kind, uint64_t seed, int64_t first, int64_t n_cand, int32_t n_tiles, int32_t b,
                             int32_t n_levels, hesp_cand *cands, int8_t *levels, void *stream) {
    if (n_cand < 0 || first < 0 || !levels || n_tiles < 1 || n_tiles > HESP_MAX_TILES) return HESP_ERR_ARG;
    if (kind != HESP_GEN_EXHAUSTIVE && kind != HESP_GEN_UNIFORM) return HESP_ERR_ARG;
    if (kind == HESP_GEN_UNIFORM && (n_levels < 1 || n_levels > HESP_MAX_LEVEL + 1)) return HESP_ERR_ARG;
    return launch_generate(kind, seed, first, n_cand, n_tiles, b, n_levels, cands, levels, (cudaStream_t)stream);
}

int hesp_generate_mutants(const int8_t *parents_dev, int32_t n_parents, int32_t n_base, int32_t n_levels,
                          double p_mut, uint64_t seed, int64_t first, int64_t n, int8_t *levels_dev, void *stream) {
    if (!parents_dev || !levels_dev || n_parents < 1 || n_base < 1 || n_levels < 1 || n_levels > 127 || n < 0 ||
        first < 0 || !(p_mut >= 0.0 && p_mut <= 1.0))
        return HESP_ERR_ARG;
    const uint32_t p_num = (uint32_t)(p_mut * 65536.0 + 0.5);
    return launch_mutate(parents_dev, n_parents, n_base, n_levels, p_num, seed, first, n, levels_dev,
                         (cudaStream_t)stream);
}

int hesp_sort_cands_workspace_size(int64_t n_cand, size_t *bytes_out) {
    if (n_cand < 0 || !bytes_out) return HESP_ERR_ARG;
    *bytes_out = (size_t)(65536 + n_cand) * 4;
    return HESP_OK;
}

int hesp_sort_cands_by_size(const hesp_cand *cands_dev, const int8_t *levels_dev, int64_t n_cand,
                            hesp_cand *sorted_dev, int32_t *perm_dev, void *workspace_dev, size_t workspace_bytes,
                            void *stream) {
    if (!cands_dev || !levels_dev || !sorted_dev || !workspace_dev || n_cand < 0 || n_cand > INT32_MAX)
        return HESP_ERR_ARG;
    if (workspace_bytes < (size_t)(65536 + n_cand) * 4 || ((uintptr_t)workspace_dev & 3)) return HESP_ERR_ARG;
    return launch_sort_by_size(cands_dev, levels_dev, n_cand, sorted_dev, perm_dev, workspace_dev,
                               (cudaStream_t)stream);
}

int hesp_generate_uneven(uint64_t seed, int64_t first, int64_t n_cand, hesp_cand *cands, int8_t *levels,
                         int64_t levels_cap, int64_t *levels_used, void *stream) {
    if (n_cand < 0 || first < 0 || !cands || !levels || !levels_used || levels_cap < 0) return HESP_ERR_ARG;
    return launch_generate_uneven(seed, first, n_cand, cands, levels, levels_cap, levels_used, (cudaStream_t)stream);
}

}  // extern "C"
