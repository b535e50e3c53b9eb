/*
 * hesp_oracle.c -- plain, slow, single-threaded CPU oracle of the HeSP
 * scheduling-partitioning simulation (Rey, Igual, Prieto-Matias, HeSP,
 * arXiv 1602.05510).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no source, header, table or helper with the
 * CUDA library; it is written from the paper's text (and, where the paper is
 * silent, from the readings stated next to each rule below), in the order the
 * paper describes the method, without blocking or fusion, so that it can be
 * checked against the paper by eye.
 *
 * What it computes, by section of the paper:
 *   - Sec. 1.1, Fig. 1: the blocked Cholesky loop that creates the base tasks
 *     (chol, trsm, gemm, syrk on b x b tiles, upper storage A[k][j], j >= k).
 *   - Sec. 2.1 "Recursive task partitioners", Fig. 3: a task is replaced in
 *     place by the tasks of its own 2x2 blocked algorithm; recursion gives a
 *     hierarchical DAG.  The partition is given as a preorder split tree.
 *   - Sec. 2.1 (RaW / WaR / WaW): dependences from overlapping data regions,
 *     both as the plain all-pairs definition and via per-atom last writers.
 *   - Sec. 2.1 "Performance and data transfer models": integer task times
 *     ceil(flops / rate) and transfer times latency + ceil(bytes / bw).
 *   - Sec. 2.1 "Task and data scheduling heuristics": FCFS or priority-list
 *     (PL) task order at release time with the EFT-P, EIT-P, F-P or R-P
 *     processor choice, accelerator memories as write-back, write-through or
 *     write-around software caches of host memory (MSI), transfers issued
 *     at scheduling time (prefetch).
 *   - Sec. 2 (problem statement): output is the task set, the task-to-
 *     processor mapping, and the makespan.
 *
 * All simulated times are int64 nanoseconds; no floating point is used.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_CAPACITY (-2)
#define OR_ERR_STATE (-5)

enum { OP_CHOL = 0, OP_TRSM = 1, OP_SYRK = 2, OP_GEMM = 3 };

/* flops of a task on a bs x bs block = coef * bs^3 / 3
 * (chol bs^3/3, trsm bs^3, syrk bs^3, gemm 2 bs^3). */
static const int64_t FLOP_COEF3[4] = {1, 3, 3, 6};

#define OR_MAX_TYPES 8
#define OR_MAX_PROCS 64
#define OR_MAX_MEMS 8
#define OR_MAX_OVR 256

/* Platform: memory spaces, processor types with performance models, the
 * processors (each bound to one memory) and one transfer model shared by
 * every pair of memories (Sec. 2: platform description). */
typedef struct {
    int32_t n_mem;
    int32_t n_types;
    int64_t peak_gflops[OR_MAX_TYPES];
    int64_t h[OR_MAX_TYPES];
    int32_t eff_pct[OR_MAX_TYPES][4]; /* per op: chol, trsm, syrk, gemm */
    int32_t n_procs;
    int32_t proc_mem[OR_MAX_PROCS];
    int32_t proc_type[OR_MAX_PROCS];
    int64_t xfer_latency_ns;
    int64_t bytes_per_elem;
    int64_t bw_bytes_per_ns;
    /* measured-model overrides: (op, type, block) -> ns */
    int32_t n_ovr;
    int32_t ovr_op[OR_MAX_OVR], ovr_type[OR_MAX_OVR];
    int64_t ovr_bs[OR_MAX_OVR], ovr_ns[OR_MAX_OVR];
    /* scheduling heuristics (Sec. 2.1): task order 0 = FCFS, 1 = PL;
     * processor selection 0 = EFT-P, 1 = EIT-P, 2 = F-P, 3 = R-P */
    int32_t order;
    int32_t select;
    uint64_t rp_seed; /* R-P: seed of the per-task processor draws */
    /* caching of accelerator memories (Sec. 2.1): 0 = write-back (WB),
     * 1 = write-through (WT), 2 = write-around (WA) */
    int32_t cache;
    /* network topology: with use_links, a message from memory s to memory d
     * takes link_lat[s][d] + ceil(bytes / link_bw[s][d]) ns (a direct link per
     * ordered pair, no contention); otherwise every pair uses the scalars */
    int32_t use_links;
    int64_t link_lat[OR_MAX_MEMS][OR_MAX_MEMS];
    int64_t link_bw[OR_MAX_MEMS][OR_MAX_MEMS];
    /* finite memory spaces (Sec. 2): capacity of each accelerator memory in
     * bytes, 0 = unbounded; host memory (0) is always unbounded */
    int64_t cap_bytes[OR_MAX_MEMS];
} or_platform;

/* A square data region in element coordinates of the full matrix. */
typedef struct {
    int64_t r0, c0, sz;
} or_region;

/* A task: its operation, its block size, its depth in the partition
 * hierarchy, and its regions.  The last region is the one written (read-
 * modify-write); the others are read only. */
typedef struct {
    int32_t op;
    int32_t depth; /* number of task clusters containing it */
    int32_t base;  /* base task it descends from */
    int32_t nreg;
    int64_t bs;
    or_region reg[3];
} or_task;

typedef struct {
    int32_t n;
    int32_t cap;
    or_task *t;
} or_dag;

/* ------------------------------------------------------------------ */
/* Performance and transfer models                                     */
/* ------------------------------------------------------------------ */

static int64_t ceil_div128(__int128 a, __int128 b) {
    __int128 q = a / b;
    if (q * b < a) q += 1;
    return (int64_t)q;
}

/* Task time = ceil(flops / rate), with
 *   flops = coef * bs^3 / 3
 *   rate  = peak * (eff_pct / 100) * bs^2 / (bs^2 + h^2)   [GFLOP/s = flop/ns]
 * evaluated as one exact rational. */
int64_t or_exec_ns(const or_platform *p, int32_t op, int32_t type, int64_t bs) {
    for (int i = 0; i < p->n_ovr; i++)
        if (p->ovr_op[i] == op && p->ovr_type[i] == type && p->ovr_bs[i] == bs)
            return p->ovr_ns[i];
    __int128 flops_num = (__int128)FLOP_COEF3[op] * bs * bs * bs; /* over 3 */
    __int128 flops_den = 3;
    __int128 rate_num = (__int128)p->peak_gflops[type] * p->eff_pct[type][op] * bs * bs;
    __int128 rate_den = (__int128)100 * (bs * bs + p->h[type] * p->h[type]);
    /* flops / rate = (flops_num * rate_den) / (flops_den * rate_num) */
    return ceil_div128(flops_num * rate_den, flops_den * rate_num);
}

/* Transfer of E elements between two memory spaces. */
int64_t or_xfer_ns(const or_platform *p, int64_t elems) {
    __int128 bytes = (__int128)elems * p->bytes_per_elem;
    return p->xfer_latency_ns + ceil_div128(bytes, p->bw_bytes_per_ns);
}

/* A message of `elems` elements from memory s to memory d. */
int64_t or_xfer_pair_ns(const or_platform *p, int32_t s, int32_t d, int64_t elems) {
    if (!p->use_links) return or_xfer_ns(p, elems);
    __int128 bytes = (__int128)elems * p->bytes_per_elem;
    return p->link_lat[s][d] + ceil_div128(bytes, p->link_bw[s][d]);
}

/* ------------------------------------------------------------------ */
/* DAG construction: base loop of Fig. 1 plus recursive 2x2 partitions */
/* ------------------------------------------------------------------ */

static int dag_push(or_dag *d, const or_task *t) {
    if (d->n >= d->cap) return OR_ERR_CAPACITY;
    d->t[d->n++] = *t;
    return OR_OK;
}

/* Block (p, q) of region r cut into k x k square blocks. */
static or_region part(or_region r, int64_t k, int64_t p, int64_t q) {
    or_region o;
    int64_t h = r.sz / k;
    o.r0 = r.r0 + p * h;
    o.c0 = r.c0 + q * h;
    o.sz = h;
    return o;
}

static int emit(or_dag *d, const int8_t *code, int64_t code_len, int64_t *pos,
                int32_t op, int32_t depth, int32_t base, or_region a, or_region b, or_region c);

/* Emit a task, or, when the split tree says so, the tasks of its blocked
 * algorithm in their program order (each of them again subject to the tree).
 * Sec. 2.1: a partitioner is the task's blocked algorithm with a partition
 * parameter p; the new tasks work on blocks of p times the task's block
 * size.  A split code value s >= 1 takes p = 1 / (s + 1): the task's blocks
 * are cut into k x k blocks, k = s + 1 (k = 2 is the 2x2 partition of
 * Fig. 3; k = 3 gives the non-dyadic tilings of Fig. 4).
 * Region arguments: chol(A=a); trsm(T=a, B=b); syrk(A=a, C=b); gemm(A=a, B=b, C=c).
 *
 *   chol(A):   the loop of Fig. 1 on the k x k blocks of A:
 *              for p: chol(App); for q > p: trsm(App -> Apq);
 *                     for i > p: { for q > i: gemm(Api, Apq -> Aiq); syrk(Api -> Aii) }
 *   trsm(T,B): B := T^-T B, T upper triangular, one block row at a time:
 *              for p: { for c: trsm(Tpp -> Bpc);
 *                       for i > p: for c: gemm(Tpi, Bpc -> Bic) }
 *   syrk(A,C): C -= A^T A on the upper part of C, in the inner order of Fig. 1:
 *              for p: for i: { for j > i: gemm(Api, Apj -> Cij); syrk(Api -> Cii) }
 *   gemm(A,B,C): C -= A^T B: for p, for i, for j: gemm(Api, Bpj -> Cij)
 * For k = 2 these are, in order: chol(A00) trsm(A00->A01) syrk(A01->A11)
 * chol(A11); trsm(T00->B00) trsm(T00->B01) gemm(T01,B00->B10)
 * gemm(T01,B01->B11) trsm(T11->B10) trsm(T11->B11); per p: gemm(Ap0,Ap1->C01)
 * syrk(Ap0->C00) syrk(Ap1->C11); and the eight gemms in p, i, j order.
 */
static int emit(or_dag *d, const int8_t *code, int64_t code_len, int64_t *pos,
                int32_t op, int32_t depth, int32_t base, or_region a, or_region b, or_region c) {
    if (*pos >= code_len) return OR_ERR_ARG;
    int8_t split = code[(*pos)++];
    int rc = OR_OK;
    if (!split) {
        or_task t;
        memset(&t, 0, sizeof t);
        t.op = op;
        t.depth = depth;
        t.base = base;
        t.bs = a.sz;
        if (op == OP_CHOL) {
            t.nreg = 1;
            t.reg[0] = a;
        } else if (op == OP_TRSM || op == OP_SYRK) {
            t.nreg = 2;
            t.reg[0] = a;
            t.reg[1] = b;
        } else {
            t.nreg = 3;
            t.reg[0] = a;
            t.reg[1] = b;
            t.reg[2] = c;
        }
        return dag_push(d, &t);
    }
    int64_t k = (int64_t)split + 1;
    if (split < 0 || a.sz % k != 0) return OR_ERR_ARG;
    or_region z = {0, 0, 0};
    int nd = depth + 1;
    switch (op) {
    case OP_CHOL:
        for (int64_t p = 0; p < k; p++) {
            if ((rc = emit(d, code, code_len, pos, OP_CHOL, nd, base, part(a, k, p, p), z, z))) return rc;
            for (int64_t q = p + 1; q < k; q++)
                if ((rc = emit(d, code, code_len, pos, OP_TRSM, nd, base, part(a, k, p, p), part(a, k, p, q), z)))
                    return rc;
            for (int64_t i = p + 1; i < k; i++) {
                for (int64_t q = i + 1; q < k; q++)
                    if ((rc = emit(d, code, code_len, pos, OP_GEMM, nd, base, part(a, k, p, i), part(a, k, p, q),
                                   part(a, k, i, q))))
                        return rc;
                if ((rc = emit(d, code, code_len, pos, OP_SYRK, nd, base, part(a, k, p, i), part(a, k, i, i), z)))
                    return rc;
            }
        }
        break;
    case OP_TRSM:
        for (int64_t p = 0; p < k; p++) {
            for (int64_t cc = 0; cc < k; cc++)
                if ((rc = emit(d, code, code_len, pos, OP_TRSM, nd, base, part(a, k, p, p), part(b, k, p, cc), z)))
                    return rc;
            for (int64_t i = p + 1; i < k; i++)
                for (int64_t cc = 0; cc < k; cc++)
                    if ((rc = emit(d, code, code_len, pos, OP_GEMM, nd, base, part(a, k, p, i), part(b, k, p, cc),
                                   part(b, k, i, cc))))
                        return rc;
        }
        break;
    case OP_SYRK:
        for (int64_t p = 0; p < k; p++)
            for (int64_t i = 0; i < k; i++) {
                for (int64_t j = i + 1; j < k; j++)
                    if ((rc = emit(d, code, code_len, pos, OP_GEMM, nd, base, part(a, k, p, i), part(a, k, p, j),
                                   part(b, k, i, j))))
                        return rc;
                if ((rc = emit(d, code, code_len, pos, OP_SYRK, nd, base, part(a, k, p, i), part(b, k, i, i), z)))
                    return rc;
            }
        break;
    case OP_GEMM:
        for (int64_t p = 0; p < k; p++)
            for (int64_t i = 0; i < k; i++)
                for (int64_t j = 0; j < k; j++)
                    if ((rc = emit(d, code, code_len, pos, OP_GEMM, nd, base, part(a, k, p, i), part(b, k, p, j),
                                   part(c, k, i, j))))
                        return rc;
        break;
    default:
        return OR_ERR_ARG;
    }
    return OR_OK;
}

static or_region tile(int64_t i, int64_t j, int64_t b) {
    or_region r = {i * b, j * b, b};
    return r;
}

/* Base task list in the loop order of Fig. 1 (upper storage):
 *   for k: chol(k); for j>k: trsm(k,j); for i>k: { for j>i: gemm(k,i,j); syrk(k,i) }
 * Each base task is then expanded following the split tree `code`
 * (preorder, 1 = partition this task, 0 = keep it). */
static int build_dag(int32_t n, int64_t b, const int8_t *code, int64_t code_len, or_dag *d) {
    int64_t pos = 0;
    int32_t base = 0;
    int rc;
    or_region z = {0, 0, 0};
    for (int32_t k = 0; k < n; k++) {
        if ((rc = emit(d, code, code_len, &pos, OP_CHOL, 0, base++, tile(k, k, b), z, z))) return rc;
        for (int32_t j = k + 1; j < n; j++)
            if ((rc = emit(d, code, code_len, &pos, OP_TRSM, 0, base++, tile(k, k, b), tile(k, j, b), z))) return rc;
        for (int32_t i = k + 1; i < n; i++) {
            for (int32_t j = i + 1; j < n; j++)
                if ((rc = emit(d, code, code_len, &pos, OP_GEMM, 0, base++, tile(k, i, b), tile(k, j, b), tile(i, j, b))))
                    return rc;
            if ((rc = emit(d, code, code_len, &pos, OP_SYRK, 0, base++, tile(k, i, b), tile(i, i, b), z))) return rc;
        }
    }
    if (pos != code_len) return OR_ERR_ARG;
    return OR_OK;
}

/* Number of base tasks of Fig. 1 for n tiles, by enumeration. */
int64_t or_base_count(int32_t n) {
    int64_t c = 0;
    for (int32_t k = 0; k < n; k++) {
        c += 1;
        for (int32_t j = k + 1; j < n; j++) c += 1;
        for (int32_t i = k + 1; i < n; i++) {
            for (int32_t j = i + 1; j < n; j++) c += 1;
            c += 1;
        }
    }
    return c;
}

/* Ops of the base tasks, in order (for building split codes). */
int or_base_ops(int32_t n, int32_t *ops_out) {
    int64_t c = 0;
    for (int32_t k = 0; k < n; k++) {
        ops_out[c++] = OP_CHOL;
        for (int32_t j = k + 1; j < n; j++) ops_out[c++] = OP_TRSM;
        for (int32_t i = k + 1; i < n; i++) {
            for (int32_t j = i + 1; j < n; j++) ops_out[c++] = OP_GEMM;
            ops_out[c++] = OP_SYRK;
        }
    }
    return OR_OK;
}

/* Preorder split code of a task split uniformly `level` times. */
static int64_t uniform_code(int32_t op, int32_t level, int8_t *out, int64_t pos, int64_t cap) {
    if (pos >= cap) return -1;
    if (level == 0) {
        out[pos++] = 0;
        return pos;
    }
    out[pos++] = 1;
    static const int32_t chol_kids[4] = {OP_CHOL, OP_TRSM, OP_SYRK, OP_CHOL};
    static const int32_t trsm_kids[6] = {OP_TRSM, OP_TRSM, OP_GEMM, OP_GEMM, OP_TRSM, OP_TRSM};
    static const int32_t syrk_kids[6] = {OP_GEMM, OP_SYRK, OP_SYRK, OP_GEMM, OP_SYRK, OP_SYRK};
    const int32_t *kids;
    int nk;
    if (op == OP_CHOL) { kids = chol_kids; nk = 4; }
    else if (op == OP_TRSM) { kids = trsm_kids; nk = 6; }
    else if (op == OP_SYRK) { kids = syrk_kids; nk = 6; }
    else { kids = NULL; nk = 8; }
    for (int i = 0; i < nk; i++) {
        pos = uniform_code(kids ? kids[i] : OP_GEMM, level - 1, out, pos, cap);
        if (pos < 0) return -1;
    }
    return pos;
}

/* Split code for the "one level per base task" partitions of the workloads:
 * base task t is split uniformly levels[t] times. Returns the code length or
 * a negative error. */
int64_t or_levels_to_code(int32_t n, const int8_t *levels, int8_t *code, int64_t cap) {
    int64_t nb = or_base_count(n);
    int32_t *ops = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    if (!ops) return OR_ERR_CAPACITY;
    or_base_ops(n, ops);
    int64_t pos = 0;
    for (int64_t t = 0; t < nb; t++) {
        if (levels[t] < 0) { free(ops); return OR_ERR_ARG; }
        pos = uniform_code(ops[t], levels[t], code, pos, cap);
        if (pos < 0) { free(ops); return OR_ERR_CAPACITY; }
    }
    free(ops);
    return pos;
}

/* ------------------------------------------------------------------ */
/* Exported DAG queries                                                */
/* ------------------------------------------------------------------ */

/* Expand the DAG for a split code. Per task outputs (length = cap):
 *   op, depth, base, nreg, bs, and regions as 9 int64 (r0,c0,sz) x 3.
 * Returns the task count or a negative error. */
int64_t or_expand(int32_t n, int64_t b, const int8_t *code, int64_t code_len, int64_t cap,
                  int32_t *op, int32_t *depth, int32_t *base, int32_t *nreg, int64_t *bs, int64_t *regs) {
    if (n < 1 || b < 1) return OR_ERR_ARG;
    or_dag d;
    d.n = 0;
    d.cap = (int32_t)cap;
    d.t = (or_task *)malloc(sizeof(or_task) * (size_t)(cap > 0 ? cap : 1));
    if (!d.t) return OR_ERR_CAPACITY;
    int rc = build_dag(n, b, code, code_len, &d);
    if (rc) { free(d.t); return rc; }
    for (int32_t i = 0; i < d.n; i++) {
        op[i] = d.t[i].op;
        depth[i] = d.t[i].depth;
        base[i] = d.t[i].base;
        nreg[i] = d.t[i].nreg;
        bs[i] = d.t[i].bs;
        for (int r = 0; r < 3; r++) {
            regs[i * 9 + r * 3 + 0] = d.t[i].reg[r].r0;
            regs[i * 9 + r * 3 + 1] = d.t[i].reg[r].c0;
            regs[i * 9 + r * 3 + 2] = d.t[i].reg[r].sz;
        }
    }
    int64_t nt = d.n;
    free(d.t);
    return nt;
}

static int overlap(or_region x, or_region y) {
    if (x.sz == 0 || y.sz == 0) return 0;
    return x.r0 < y.r0 + y.sz && y.r0 < x.r0 + x.sz && x.c0 < y.c0 + y.sz && y.c0 < x.c0 + x.sz;
}

/* Dependence of task j on an earlier task i (Sec. 2.1: RaW, WaR, WaW):
 * j depends on i iff  W_i meets (R_j u W_j)  or  R_i meets W_j. */
static int depends(const or_task *i, const or_task *j) {
    or_region wi = i->reg[i->nreg - 1];
    or_region wj = j->reg[j->nreg - 1];
    for (int r = 0; r < j->nreg; r++)
        if (overlap(wi, j->reg[r])) return 1;
    for (int r = 0; r < i->nreg - 1; r++)
        if (overlap(i->reg[r], wj)) return 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Dependences via atoms                                               */
/* ------------------------------------------------------------------ */

/* The matrix is cut into square atoms of side a (b / 2^atom_level for the
 * dyadic partitions, b / lcm of the factors for the one-level k-way ones);
 * every region of the DAG must be a union of atoms.
 * For task j, in creation order, and every atom x of its regions:
 *   RaW / WaW: j depends on the last writer of x;
 *   WaR: if j writes x, j depends on every reader of x since its last write.
 * Then j becomes the last writer of its written atoms and a reader of the
 * others. */
typedef struct {
    int32_t n;
    int32_t cap;
    int32_t *v;
} ivec;

static int ivec_push(ivec *v, int32_t x) {
    if (v->n == v->cap) {
        int32_t nc = v->cap ? v->cap * 2 : 4;
        int32_t *nv = (int32_t *)realloc(v->v, sizeof(int32_t) * (size_t)nc);
        if (!nv) return OR_ERR_CAPACITY;
        v->v = nv;
        v->cap = nc;
    }
    v->v[v->n++] = x;
    return OR_OK;
}

typedef struct {
    int64_t a;    /* atom side in elements */
    int64_t grid; /* atoms per matrix side */
} atom_grid;

static int64_t atom_id(const atom_grid *g, int64_t ar, int64_t ac) { return ar * g->grid + ac; }

/* The atoms of a region, listed row by row. Returns count. */
static int64_t region_atoms(const atom_grid *g, or_region r, int64_t *out) {
    int64_t k = 0;
    int64_t s = r.sz / g->a;
    for (int64_t i = 0; i < s; i++)
        for (int64_t j = 0; j < s; j++) out[k++] = atom_id(g, r.r0 / g->a + i, r.c0 / g->a + j);
    return k;
}

/* Build predecessor lists (CSR by task) from atoms. Predecessors of each task
 * are listed once each, in ascending order. */
static int atom_deps(const or_dag *d, const atom_grid *g, int64_t **pred_off_out, int32_t **preds_out,
                     int32_t *war_edges) {
    int64_t natoms = g->grid * g->grid;
    int32_t *last_writer = (int32_t *)malloc(sizeof(int32_t) * (size_t)natoms);
    ivec *readers = (ivec *)calloc((size_t)natoms, sizeof(ivec));
    int64_t *pred_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(d->n + 1));
    int8_t *mark = (int8_t *)calloc((size_t)d->n, 1);
    ivec preds = {0, 0, NULL};
    ivec cur = {0, 0, NULL};
    int64_t maxatoms = 0;
    for (int32_t j = 0; j < d->n; j++) {
        int64_t s = d->t[j].bs / g->a;
        if (3 * s * s > maxatoms) maxatoms = 3 * s * s;
    }
    int64_t *ax = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxatoms + 1));
    int rc = OR_OK;
    if (!last_writer || !readers || !pred_off || !mark || !ax) { rc = OR_ERR_CAPACITY; goto out; }
    for (int64_t x = 0; x < natoms; x++) last_writer[x] = -1;
    *war_edges = 0;
    pred_off[0] = 0;
    for (int32_t j = 0; j < d->n; j++) {
        const or_task *t = &d->t[j];
        cur.n = 0;
        for (int r = 0; r < t->nreg; r++) {
            int is_w = (r == t->nreg - 1);
            int64_t na = region_atoms(g, t->reg[r], ax);
            for (int64_t q = 0; q < na; q++) {
                int64_t x = ax[q];
                int32_t w = last_writer[x];
                if (w >= 0 && !mark[w]) { mark[w] = 1; if ((rc = ivec_push(&cur, w))) goto out; }
                if (is_w) {
                    for (int32_t e = 0; e < readers[x].n; e++) {
                        int32_t rd = readers[x].v[e];
                        if (rd != j && !mark[rd]) {
                            mark[rd] = 1;
                            (*war_edges)++;
                            if ((rc = ivec_push(&cur, rd))) goto out;
                        }
                    }
                }
            }
        }
        /* ascending order, then clear marks */
        for (int32_t a1 = 1; a1 < cur.n; a1++) {
            int32_t v = cur.v[a1];
            int32_t a2 = a1 - 1;
            while (a2 >= 0 && cur.v[a2] > v) { cur.v[a2 + 1] = cur.v[a2]; a2--; }
            cur.v[a2 + 1] = v;
        }
        for (int32_t e = 0; e < cur.n; e++) {
            mark[cur.v[e]] = 0;
            if ((rc = ivec_push(&preds, cur.v[e]))) goto out;
        }
        pred_off[j + 1] = preds.n;
        /* update the per-atom state after all reads of this task */
        for (int r = 0; r < t->nreg; r++) {
            int is_w = (r == t->nreg - 1);
            int64_t na = region_atoms(g, t->reg[r], ax);
            for (int64_t q = 0; q < na; q++) {
                int64_t x = ax[q];
                if (is_w) {
                    last_writer[x] = j;
                    readers[x].n = 0;
                } else {
                    if ((rc = ivec_push(&readers[x], j))) goto out;
                }
            }
        }
    }
out:
    if (readers) {
        for (int64_t x = 0; x < natoms; x++) free(readers[x].v);
        free(readers);
    }
    free(last_writer);
    free(mark);
    free(ax);
    free(cur.v);
    if (rc) {
        free(pred_off);
        free(preds.v);
        return rc;
    }
    *pred_off_out = pred_off;
    *preds_out = preds.v ? preds.v : (int32_t *)malloc(sizeof(int32_t));
    return OR_OK;
}

/* All-pairs predecessor lists straight from the definition (O(T^2)). */
static int allpairs_deps(const or_dag *d, int64_t **pred_off_out, int32_t **preds_out) {
    int64_t *pred_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(d->n + 1));
    ivec preds = {0, 0, NULL};
    if (!pred_off) return OR_ERR_CAPACITY;
    pred_off[0] = 0;
    for (int32_t j = 0; j < d->n; j++) {
        for (int32_t i = 0; i < j; i++)
            if (depends(&d->t[i], &d->t[j]))
                if (ivec_push(&preds, i)) { free(pred_off); free(preds.v); return OR_ERR_CAPACITY; }
        pred_off[j + 1] = preds.n;
    }
    *pred_off_out = pred_off;
    *preds_out = preds.v ? preds.v : (int32_t *)malloc(sizeof(int32_t));
    return OR_OK;
}

static int make_dag(int32_t n, int64_t b, const int8_t *code, int64_t code_len, int64_t cap, or_dag *d) {
    d->n = 0;
    d->cap = (int32_t)cap;
    d->t = (or_task *)malloc(sizeof(or_task) * (size_t)(cap > 0 ? cap : 1));
    if (!d->t) return OR_ERR_CAPACITY;
    int rc = build_dag(n, b, code, code_len, d);
    if (rc) { free(d->t); d->t = NULL; }
    return rc;
}

/* Atoms of side `side` elements: every region of the DAG must be a union of
 * them (side divides b and every region's offsets and size). */
static int check_atoms(const or_dag *d, int64_t b, int64_t side, atom_grid *g, int32_t n) {
    if (side < 1 || b % side != 0) return OR_ERR_ARG;
    g->a = side;
    g->grid = (int64_t)n * (b / side);
    for (int32_t j = 0; j < d->n; j++)
        for (int r = 0; r < d->t[j].nreg; r++) {
            or_region x = d->t[j].reg[r];
            if (x.sz % g->a || x.r0 % g->a || x.c0 % g->a) return OR_ERR_ARG;
        }
    return OR_OK;
}

/* Dependence lists for a split code. mode 0: all pairs (definition);
 * mode 1: atoms of side atom_side.  Output: pred_off[T+1], preds[cap_e].
 * Returns the edge count, or a negative error. war_out: WaR edges found. */
int64_t or_deps_side(int32_t n, int64_t b, const int8_t *code, int64_t code_len, int64_t cap_t, int32_t mode,
                     int64_t atom_side, int64_t cap_e, int64_t *pred_off, int32_t *preds, int32_t *war_out) {
    or_dag d;
    int rc = make_dag(n, b, code, code_len, cap_t, &d);
    if (rc) return rc;
    int64_t *po = NULL;
    int32_t *pv = NULL;
    int32_t war = 0;
    if (mode == 0) {
        rc = allpairs_deps(&d, &po, &pv);
    } else {
        atom_grid g;
        rc = check_atoms(&d, b, atom_side, &g, n);
        if (!rc) rc = atom_deps(&d, &g, &po, &pv, &war);
    }
    if (rc) { free(d.t); return rc; }
    int64_t ne = po[d.n];
    if (ne > cap_e) { free(d.t); free(po); free(pv); return OR_ERR_CAPACITY; }
    memcpy(pred_off, po, sizeof(int64_t) * (size_t)(d.n + 1));
    memcpy(preds, pv, sizeof(int32_t) * (size_t)ne);
    if (war_out) *war_out = war;
    free(d.t);
    free(po);
    free(pv);
    return ne;
}

/* or_deps with atoms of side b / 2^atom_level. */
int64_t or_deps(int32_t n, int64_t b, const int8_t *code, int64_t code_len, int64_t cap_t, int32_t mode,
                int32_t atom_level, int64_t cap_e, int64_t *pred_off, int32_t *preds, int32_t *war_out) {
    if (mode != 0 && (atom_level < 0 || atom_level > 20 || b % ((int64_t)1 << atom_level) != 0)) return OR_ERR_ARG;
    return or_deps_side(n, b, code, code_len, cap_t, mode, mode == 0 ? 1 : b >> atom_level, cap_e, pred_off, preds,
                        war_out);
}

/* ------------------------------------------------------------------ */
/* Event-driven FCFS + EFT-P simulation with MSI write-back coherence   */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t makespan;
    int64_t n_tasks;
    int64_t n_events;     /* distinct completion times processed */
    int64_t n_transfers;  /* messages issued */
    int64_t xfer_elems;   /* elements moved */
    int64_t atom_visits;  /* sum over tasks of atoms in their regions */
    int64_t evicted;      /* atoms evicted from finite memories */
    int64_t written_back; /* of those, atoms written back to host memory */
} or_stats;

/* State of one simulation, shared by the task-order loops below. */
typedef struct {
    const or_platform *pl;
    const or_dag *d;
    const atom_grid *g;
    int32_t M, P;
    uint8_t *valid;
    int64_t *vfrom;
    int64_t *avail;
    const int8_t *mem_used;
    int64_t *ax;
    int32_t *axw;
    int32_t *src;
    or_stats *st;
    int64_t *use;                     /* per atom x memory: latest finish of a task that used it there */
    int8_t bounded[OR_MAX_MEMS];      /* finite memory */
    int64_t cap_atoms[OR_MAX_MEMS];   /* its capacity in atoms (whole atoms only) */
    uint8_t *wb;                      /* per atom: written back by the current eviction */
    int16_t *proc_out;
    int64_t *start_out, *finish_out;
    int32_t *order_out;
    int64_t *issue_out;
    int32_t n_sched;
    int64_t finish_j; /* finish time of the task just scheduled */
} sched_state;

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the stream value for
 * counter (c, k) is the published output function applied to
 * seed + ((c << 32) + k + 1) * 0x9E3779B97F4A7C15; a draw in [0, m) takes
 * the high 32 bits times m, shifted down by 32 (Lemire). */
static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint32_t sm64_draw(uint64_t seed, uint64_t c, uint64_t k, uint32_t m) {
    uint64_t u = sm64_mix(seed + ((c << 32) + k + 1) * 0x9E3779B97F4A7C15ULL);
    return (uint32_t)(((u >> 32) * (uint64_t)m) >> 32);
}

/* Is some processor idle at t (nothing running or queued on it after t)? */
static int any_idle(const int64_t *avail, int32_t P, int64_t t) {
    for (int p = 0; p < P; p++)
        if (avail[p] <= t) return 1;
    return 0;
}

/* Schedule task j at time t (see the rules above or_simulate). */
static int schedule_task(sched_state *S, int32_t j, int64_t t) {
    const or_platform *pl = S->pl;
    const or_task *tk = &S->d->t[j];
    const atom_grid *g = S->g;
    const int32_t M = S->M, P = S->P;
    uint8_t *valid = S->valid;
    int64_t *vfrom = S->vfrom;
    int64_t *ax = S->ax;
    int32_t *axw = S->axw, *src = S->src;
    /* atoms of j's regions, flagged when written */
    int64_t na = 0;
    for (int r = 0; r < tk->nreg; r++) {
        int64_t k = region_atoms(g, tk->reg[r], ax + na);
        for (int64_t e = 0; e < k; e++) axw[na + e] = (r == tk->nreg - 1);
        na += k;
    }
    S->st->atom_visits += na;
    int64_t atom_elems = g->a * g->a;
    int64_t drt[OR_MAX_MEMS];
    int64_t arrive[OR_MAX_MEMS][OR_MAX_MEMS];
    for (int m = 0; m < M; m++) {
        drt[m] = 0;
        if (!S->mem_used[m]) continue;
        int64_t elems_from[OR_MAX_MEMS], depart[OR_MAX_MEMS];
        for (int sm = 0; sm < M; sm++) {
            elems_from[sm] = 0;
            depart[sm] = t;
        }
        for (int64_t e = 0; e < na; e++) {
            int64_t x = ax[e];
            src[e * M + m] = -1;
            if (valid[x * M + m]) {
                if (vfrom[x * M + m] > drt[m]) drt[m] = vfrom[x * M + m];
            } else {
                /* the lowest memory with a copy usable at t; if there is none
                 * (under WA a block may be valid only in flight to the host),
                 * the copy usable first (ties to the lower memory) */
                int found = -1;
                for (int sm = 0; sm < M; sm++)
                    if (valid[x * M + sm] && vfrom[x * M + sm] <= t) { found = sm; break; }
                if (found < 0)
                    for (int sm = 0; sm < M; sm++)
                        if (valid[x * M + sm] && (found < 0 || vfrom[x * M + sm] < vfrom[x * M + found])) found = sm;
                if (found < 0) return OR_ERR_STATE;
                src[e * M + m] = found;
                elems_from[found] += atom_elems;
                if (vfrom[x * M + found] > depart[found]) depart[found] = vfrom[x * M + found];
            }
        }
        /* one message per source, issued when the last of its data is usable
         * there (at t under WB) */
        for (int sm = 0; sm < M; sm++) {
            arrive[m][sm] = 0;
            if (elems_from[sm] > 0) {
                arrive[m][sm] = depart[sm] + or_xfer_pair_ns(pl, sm, m, elems_from[sm]);
                if (arrive[m][sm] > drt[m]) drt[m] = arrive[m][sm];
            }
        }
    }
    /* Finite memories (reading of Sec. 2, which names finite-size memory
     * spaces but no policy): a bounded memory m can take task j at t when the
     * atoms j lacks there fit in its free space plus what it may evict --
     * atoms valid in m that j does not use and that no task in flight on m
     * still uses (use[x][m] <= t).  Processors of memories that cannot take j
     * are not candidates. */
    int feasible[OR_MAX_MEMS];
    int64_t need[OR_MAX_MEMS], room[OR_MAX_MEMS];
    int any_bounded = 0;
    for (int m = 0; m < M; m++) {
        feasible[m] = 1;
        need[m] = room[m] = 0;
        if (!S->mem_used[m] || !S->bounded[m]) continue;
        any_bounded = 1;
        for (int64_t e = 0; e < na; e++) need[m] += !valid[ax[e] * M + m];
        int64_t occ = 0, evictable = 0;
        for (int64_t x = 0; x < g->grid * g->grid; x++) {
            if (!valid[x * M + m]) continue;
            occ++;
            int mine = 0;
            for (int64_t e = 0; e < na && !mine; e++) mine = ax[e] == x;
            if (!mine && S->use[x * M + m] <= t) evictable++;
        }
        room[m] = S->cap_atoms[m] - occ;
        feasible[m] = need[m] <= room[m] + evictable;
    }
    /* processor selection, ties to the lowest id:
     *   EFT-P: the earliest finish time max(t, avail, DRT) + exec;
     *   EIT-P: the processor that becomes idle first, max(t, avail);
     *   F-P:   among the processors idle at t, the fastest for this task;
     *   R-P:   among the processors idle at t, the k-th in id order, k drawn
     *          uniformly from the SplitMix64 stream (rp_seed, task id j). */
    int32_t n_idle = 0, pick = -1;
    if (pl->select >= 2) {
        for (int p = 0; p < P; p++)
            if (S->avail[p] <= t) n_idle++;
        if (n_idle == 0) return OR_ERR_STATE;
        if (pl->select == 3) pick = (int32_t)sm64_draw(pl->rp_seed, (uint64_t)j, 0, (uint32_t)n_idle);
    }
    int32_t best = -1, idle_seen = 0;
    int64_t best_key = 0, best_eft = 0, best_exec = 0;
    for (int p = 0; p < P; p++) {
        if (pl->select >= 2 && S->avail[p] > t) continue;
        if (!feasible[pl->proc_mem[p]]) continue;
        int64_t ready = t;
        if (S->avail[p] > ready) ready = S->avail[p];
        int64_t idle = ready;
        if (drt[pl->proc_mem[p]] > ready) ready = drt[pl->proc_mem[p]];
        int64_t ex = or_exec_ns(pl, tk->op, pl->proc_type[p], tk->bs);
        int64_t eft = ready + ex;
        int64_t key;
        if (pl->select == 0) key = eft;
        else if (pl->select == 1) key = idle;
        else if (pl->select == 2) key = ex;
        else key = (idle_seen == pick) ? 0 : 1;
        idle_seen++;
        if (best < 0 || key < best_key) { best = p; best_key = key; best_eft = eft; best_exec = ex; }
    }
    if (best < 0) return OR_ERR_CAPACITY; /* no memory can take the task */
    int ms = pl->proc_mem[best];
    /* eviction from a bounded memory: the least recently used evictable atom
     * first (smallest use[x][ms], ties to the lower atom index) until the
     * missing atoms fit; an evicted atom valid in no other memory is written
     * back to host memory, all of them in one message issued at t, valid in
     * host memory from its arrival */
    if (any_bounded && S->bounded[ms] && need[ms] > room[ms]) {
        int64_t k = need[ms] - room[ms], n_wb = 0;
        for (int64_t q = 0; q < k; q++) {
            int64_t victim = -1;
            for (int64_t x = 0; x < g->grid * g->grid; x++) {
                if (!valid[x * M + ms] || S->use[x * M + ms] > t) continue;
                int mine = 0;
                for (int64_t e = 0; e < na && !mine; e++) mine = ax[e] == x;
                if (mine) continue;
                if (victim < 0 || S->use[x * M + ms] < S->use[victim * M + ms]) victim = x;
            }
            if (victim < 0) return OR_ERR_STATE;
            int elsewhere = 0;
            for (int m = 0; m < M; m++)
                if (m != ms && valid[victim * M + m]) elsewhere = 1;
            valid[victim * M + ms] = 0;
            if (!elsewhere) {
                S->wb[victim] = 1;
                n_wb++;
            }
            S->st->evicted++;
        }
        if (n_wb > 0) {
            int64_t arrive_host = t + or_xfer_pair_ns(pl, ms, 0, n_wb * atom_elems);
            for (int64_t x = 0; x < g->grid * g->grid; x++)
                if (S->wb[x]) {
                    S->wb[x] = 0;
                    valid[x * M + 0] = 1;
                    vfrom[x * M + 0] = arrive_host;
                }
            S->st->written_back += n_wb;
        }
    }
    /* commit: transfers, then write-back invalidation of written atoms */
    int64_t elems_from2[OR_MAX_MEMS];
    for (int sm = 0; sm < M; sm++) elems_from2[sm] = 0;
    for (int64_t e = 0; e < na; e++) {
        int64_t x = ax[e];
        int sm = src[e * M + ms];
        if (sm >= 0) {
            valid[x * M + ms] = 1;
            vfrom[x * M + ms] = arrive[ms][sm];
            elems_from2[sm] += atom_elems;
        }
    }
    for (int sm = 0; sm < M; sm++)
        if (elems_from2[sm] > 0) { S->st->n_transfers++; S->st->xfer_elems += elems_from2[sm]; }
    /* the written block: WB valid only in mem(p*) from the finish; WT also
     * in host memory, from the arrival of a message of the whole block issued
     * at the finish; WA (from an accelerator) only in host memory, from that
     * arrival.  Every other copy is invalidated. */
    int64_t written = 0;
    for (int64_t e = 0; e < na; e++) written += axw[e];
    const int64_t through =
        ms != 0 && pl->cache != 0 ? best_eft + or_xfer_pair_ns(pl, ms, 0, written * atom_elems) : best_eft;
    for (int64_t e = 0; e < na; e++) {
        if (!axw[e]) continue;
        int64_t x = ax[e];
        for (int m = 0; m < M; m++) valid[x * M + m] = 0;
        if (pl->cache != 2 || ms == 0) {
            valid[x * M + ms] = 1;
            vfrom[x * M + ms] = best_eft;
        }
        if (ms != 0 && pl->cache != 0) {
            valid[x * M + 0] = 1;
            vfrom[x * M + 0] = through;
        }
    }
    for (int64_t e = 0; e < na; e++)
        if (S->use[ax[e] * M + ms] < best_eft) S->use[ax[e] * M + ms] = best_eft;
    S->avail[best] = best_eft;
    S->finish_j = best_eft;
    if (S->proc_out) S->proc_out[j] = (int16_t)best;
    if (S->start_out) S->start_out[j] = best_eft - best_exec;
    if (S->finish_out) S->finish_out[j] = best_eft;
    if (S->order_out) S->order_out[S->n_sched] = j;
    if (S->issue_out) S->issue_out[j] = t;
    S->n_sched++;
    if (best_eft > S->st->makespan) S->st->makespan = best_eft;
    return OR_OK;
}

/* qsort order of the priority list: decreasing critical time, then id. */
static const int64_t *g_crit;
static int by_crit_desc(const void *a, const void *b) {
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    if (g_crit[i] != g_crit[j]) return g_crit[i] > g_crit[j] ? -1 : 1;
    return i < j ? -1 : (i > j);
}

/* Simulate one candidate.
 *   code/code_len: split tree (preorder), see or_levels_to_code
 *   atom_side:     atom side in elements (divides every region)
 *   dep_mode:      0 = all-pairs dependences, 1 = atom last-writer
 * Optional outputs (NULL to skip), per task in creation order:
 *   proc_out, start_out, finish_out, issue_out (the time at which the task
 *   was scheduled and its messages issued); order_out = task ids in the
 *   order they were scheduled.
 * The scheduling rules (Sec. 2.1, WB caching, prefetch), with task order
 * FCFS (pl->order 0) -- PL (order 1) is described at its loop below:
 *   1. t = 0; the released set holds the tasks without predecessors.
 *   2. The released tasks join the back of a first-come first-served queue
 *      in ascending task id; tasks are taken from its front and scheduled
 *      at time t.  Under EFT-P and EIT-P every task is taken at once; under
 *      F-P and R-P (which choose among idle processors only) the front task
 *      waits while no processor is idle at t, and the tasks behind it wait
 *      with it.
 *   3. If nothing is in flight, stop.  Otherwise t = the earliest finish
 *      time in flight; every task finishing at t completes, and the tasks
 *      whose predecessors have now all completed are released.
 * Scheduling task j at time t:
 *   - for each memory m holding a processor, the data ready time DRT(j, m):
 *     every atom x of j's regions that is valid in m is usable from
 *     vfrom[x][m]; every other atom is fetched from the lowest-numbered
 *     memory holding a copy usable at t (if none is, from the copy usable
 *     first); the missing atoms with the same source travel as one message,
 *     issued at t or, if later, when the last of them is usable at the
 *     source, and arrive xfer(elements) later; DRT is the latest of these
 *     times;
 *   - EFT(p) = max(t, avail[p], DRT(j, mem(p))) + exec(op, type(p), bs);
 *     EFT-P (pl->select 0): p* = argmin EFT, ties to the lowest processor
 *     id; EIT-P (select 1): p* = argmin max(t, avail[p]), ties likewise;
 *     F-P (select 2): among the processors idle at t (avail[p] <= t) the
 *     one with the least exec time, ties likewise; R-P (select 3): among
 *     the idle processors in id order, the one at a uniform draw from the
 *     SplitMix64 stream (rp_seed, j); the task still waits for its data;
 *   - commit: start = EFT - exec, avail[p*] = EFT; the fetched atoms become
 *     valid in mem(p*) from their arrival; then the written atoms are
 *     invalidated everywhere and become valid: under WB (pl->cache 0) in
 *     mem(p*) from the finish time; under WT (1) there and, when mem(p*) is
 *     not the host, in host memory from finish + xfer(block); under WA (2),
 *     when mem(p*) is not the host, only in host memory from finish +
 *     xfer(block) (else as WB).
 *   - the makespan is the largest finish time. */
int32_t or_simulate_side(const or_platform *pl, int32_t n, int64_t b, const int8_t *code, int64_t code_len,
                         int64_t cap_t, int64_t atom_side, int32_t dep_mode, int16_t *proc_out,
                         int64_t *start_out, int64_t *finish_out, int32_t *order_out, int64_t *issue_out,
                         or_stats *st) {
    if (!pl || pl->n_mem < 1 || pl->n_mem > OR_MAX_MEMS || pl->n_procs < 1 || pl->n_procs > OR_MAX_PROCS)
        return OR_ERR_ARG;
    if (pl->n_mem > 1 && pl->bw_bytes_per_ns < 1) return OR_ERR_ARG;
    if (pl->use_links)
        for (int s = 0; s < pl->n_mem; s++)
            for (int d = 0; d < pl->n_mem; d++)
                if (s != d && (pl->link_bw[s][d] < 1 || pl->link_lat[s][d] < 0)) return OR_ERR_ARG;
    for (int p = 0; p < pl->n_procs; p++)
        if (pl->proc_mem[p] < 0 || pl->proc_mem[p] >= pl->n_mem || pl->proc_type[p] < 0 ||
            pl->proc_type[p] >= pl->n_types)
            return OR_ERR_ARG;
    /* finite memories: accelerators only, with EFT-P or EIT-P (F-P and R-P
     * would also need a rule for idle processors whose memory is full) */
    int bounded = 0;
    for (int m = 0; m < pl->n_mem; m++) {
        if (pl->cap_bytes[m] < 0 || (m == 0 && pl->cap_bytes[m] != 0)) return OR_ERR_ARG;
        if (pl->cap_bytes[m] > 0) bounded = 1;
    }
    if (bounded && pl->select >= 2) return OR_ERR_ARG;
    or_dag d;
    int rc = make_dag(n, b, code, code_len, cap_t, &d);
    if (rc) return rc;
    atom_grid g;
    rc = check_atoms(&d, b, atom_side, &g, n);
    if (rc) { free(d.t); return rc; }
    int64_t *pred_off = NULL;
    int32_t *preds = NULL;
    int32_t war = 0;
    if (dep_mode == 0) rc = allpairs_deps(&d, &pred_off, &preds);
    else rc = atom_deps(&d, &g, &pred_off, &preds, &war);
    if (rc) { free(d.t); return rc; }

    const int32_t T = d.n;
    const int32_t M = pl->n_mem;
    const int32_t P = pl->n_procs;
    int64_t natoms = g.grid * g.grid;

    /* successor lists from the predecessor lists */
    int64_t *succ_off = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
    int32_t *succ = (int32_t *)malloc(sizeof(int32_t) * (size_t)(pred_off[T] + 1));
    int64_t *fill = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
    int32_t *pending = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1));
    int64_t *finish = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
    int8_t *state = (int8_t *)calloc((size_t)T + 1, 1); /* 0 waiting, 1 in flight, 2 done */
    int32_t *inflight = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1)); /* tasks in flight */
    int32_t n_inflight = 0;
    int32_t *released = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1));
    int32_t *fifo = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1)); /* FCFS queue */
    uint8_t *valid = (uint8_t *)calloc((size_t)(natoms * M), 1);
    int64_t *vfrom = (int64_t *)calloc((size_t)(natoms * M), sizeof(int64_t));
    int64_t *use = (int64_t *)malloc(sizeof(int64_t) * (size_t)(natoms * M));
    uint8_t *wbm = (uint8_t *)calloc((size_t)natoms, 1);
    int64_t maxatoms = 0;
    for (int32_t j = 0; j < T; j++) {
        int64_t s = d.t[j].bs / g.a;
        if (3 * s * s > maxatoms) maxatoms = 3 * s * s;
    }
    int64_t *ax = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxatoms + 1));
    int32_t *axw = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxatoms + 1));
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)((maxatoms + 1) * M));
    int64_t avail[OR_MAX_PROCS];
    int8_t mem_used[OR_MAX_MEMS];
    or_stats s;
    memset(&s, 0, sizeof s);
    if (!succ_off || !succ || !fill || !pending || !finish || !state || !released || !valid || !vfrom || !ax ||
        !axw || !src || !inflight || !fifo || !use || !wbm) {
        rc = OR_ERR_CAPACITY;
        goto out;
    }
    for (int32_t j = 0; j < T; j++)
        for (int64_t e = pred_off[j]; e < pred_off[j + 1]; e++) succ_off[preds[e] + 1]++;
    for (int32_t j = 0; j < T; j++) succ_off[j + 1] += succ_off[j];
    for (int32_t j = 0; j < T; j++)
        for (int64_t e = pred_off[j]; e < pred_off[j + 1]; e++) {
            int32_t i = preds[e];
            succ[succ_off[i] + fill[i]++] = j;
        }
    for (int32_t j = 0; j < T; j++) pending[j] = (int32_t)(pred_off[j + 1] - pred_off[j]);
    /* initial coherence: every atom valid in host memory from time 0 */
    for (int64_t x = 0; x < natoms; x++) {
        valid[x * M + 0] = 1;
        vfrom[x * M + 0] = 0;
    }
    for (int64_t x = 0; x < natoms * M; x++) use[x] = -1;
    for (int p = 0; p < P; p++) avail[p] = 0;
    memset(mem_used, 0, sizeof mem_used);
    for (int p = 0; p < P; p++) mem_used[pl->proc_mem[p]] = 1;

    sched_state S;
    S.pl = pl;
    S.d = &d;
    S.g = &g;
    S.M = M;
    S.P = P;
    S.valid = valid;
    S.vfrom = vfrom;
    S.avail = avail;
    S.mem_used = mem_used;
    S.ax = ax;
    S.axw = axw;
    S.src = src;
    S.st = &s;
    S.proc_out = proc_out;
    S.start_out = start_out;
    S.finish_out = finish_out;
    S.order_out = order_out;
    S.issue_out = issue_out;
    S.n_sched = 0;
    S.use = use;
    S.wb = wbm;
    for (int m = 0; m < OR_MAX_MEMS; m++) {
        int64_t ab = g.a * g.a * pl->bytes_per_elem;
        S.bounded[m] = m < M && pl->cap_bytes[m] > 0;
        S.cap_atoms[m] = S.bounded[m] ? pl->cap_bytes[m] / ab : 0;
    }
    const int waits = pl->select >= 2; /* F-P, R-P: idle processors only */
    int32_t n_done = 0;
    if (pl->order == 1) {
        /* PL: a static priority list (HEFT-like).  Critical time of a task =
         * its processing time summed over all processors (P times the mean:
         * the same order) plus the largest critical time of its successors,
         * computed backwards (creation order is topological).  Tasks are
         * scheduled in decreasing critical time, ties to the lower id, each at
         * its release time: the latest finish among its predecessors.  Under
         * F-P and R-P a task released while no processor is idle is scheduled
         * when the first one becomes idle (the least avail). */
        int64_t *crit = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
        int64_t *rel = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
        int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1));
        if (!crit || !rel || !list) {
            free(crit); free(rel); free(list);
            rc = OR_ERR_CAPACITY;
            goto out;
        }
        for (int32_t j = T - 1; j >= 0; j--) {
            int64_t w = 0, best = 0;
            for (int p = 0; p < P; p++) w += or_exec_ns(pl, d.t[j].op, pl->proc_type[p], d.t[j].bs);
            for (int64_t e = succ_off[j]; e < succ_off[j + 1]; e++)
                if (crit[succ[e]] > best) best = crit[succ[e]];
            crit[j] = w + best;
        }
        for (int32_t j = 0; j < T; j++) list[j] = j;
        g_crit = crit;
        qsort(list, (size_t)T, sizeof(int32_t), by_crit_desc);
        for (int32_t q = 0; q < T && !rc; q++) {
            int32_t j = list[q];
            int64_t t = rel[j];
            if (waits && !any_idle(avail, P, t)) {
                t = avail[0];
                for (int p = 1; p < P; p++)
                    if (avail[p] < t) t = avail[p];
            }
            rc = schedule_task(&S, j, t);
            if (rc) break;
            for (int64_t e = succ_off[j]; e < succ_off[j + 1]; e++)
                if (S.finish_j > rel[succ[e]]) rel[succ[e]] = S.finish_j;
            n_done++;
        }
        free(crit);
        free(rel);
        free(list);
        if (rc) goto out;
    } else {
        int32_t nrel = 0;
        int32_t qh = 0, qt = 0; /* the queue: fifo[qh .. qt) */
        for (int32_t j = 0; j < T; j++)
            if (pending[j] == 0) released[nrel++] = j;
        int64_t t = 0;
        for (;;) {
            /* the released tasks join the queue in ascending id */
            for (int32_t a1 = 1; a1 < nrel; a1++) {
                int32_t v = released[a1];
                int32_t a2 = a1 - 1;
                while (a2 >= 0 && released[a2] > v) { released[a2 + 1] = released[a2]; a2--; }
                released[a2 + 1] = v;
            }
            for (int32_t q = 0; q < nrel; q++) fifo[qt++] = released[q];
            nrel = 0;
            /* schedule from the front of the queue */
            while (qh < qt) {
                if (waits && !any_idle(avail, P, t)) break;
                int32_t j = fifo[qh++];
                rc = schedule_task(&S, j, t);
                if (rc) goto out;
                finish[j] = S.finish_j;
                state[j] = 1;
                inflight[n_inflight++] = j;
            }
            /* next completion time */
            int64_t tn = -1;
            for (int32_t q = 0; q < n_inflight; q++)
                if (tn < 0 || finish[inflight[q]] < tn) tn = finish[inflight[q]];
            if (tn < 0) break;
            t = tn;
            s.n_events++;
            for (int32_t q = 0; q < n_inflight;) {
                int32_t j = inflight[q];
                if (finish[j] == t) {
                    state[j] = 2;
                    n_done++;
                    for (int64_t e = succ_off[j]; e < succ_off[j + 1]; e++) {
                        int32_t sj = succ[e];
                        if (--pending[sj] == 0) released[nrel++] = sj;
                    }
                    inflight[q] = inflight[--n_inflight];
                } else {
                    q++;
                }
            }
        }
    }
    int32_t n_sched = S.n_sched;
    if (n_sched != T || n_done != T) rc = OR_ERR_STATE;
    s.n_tasks = T;
out:
    if (st) *st = s;
    free(d.t);
    free(pred_off);
    free(preds);
    free(succ_off);
    free(succ);
    free(fill);
    free(pending);
    free(finish);
    free(state);
    free(inflight);
    free(released);
    free(fifo);
    free(valid);
    free(vfrom);
    free(use);
    free(wbm);
    free(ax);
    free(axw);
    free(src);
    return rc;
}

/* or_simulate_side with atoms of side b / 2^atom_level (atom_level >= the
 * deepest split of a dyadic partition). */
int32_t or_simulate(const or_platform *pl, int32_t n, int64_t b, const int8_t *code, int64_t code_len,
                    int64_t cap_t, int32_t atom_level, int32_t dep_mode, int16_t *proc_out,
                    int64_t *start_out, int64_t *finish_out, int32_t *order_out, int64_t *issue_out,
                    or_stats *st) {
    if (atom_level < 0 || atom_level > 20 || b % ((int64_t)1 << atom_level) != 0) return OR_ERR_ARG;
    return or_simulate_side(pl, n, b, code, code_len, cap_t, b >> atom_level, dep_mode, proc_out, start_out,
                            finish_out, order_out, issue_out, st);
}

/* Convenience: one candidate given one split level per base task; the atom
 * level is the largest split level unless atom_level >= 0 is given. */
int32_t or_simulate_levels(const or_platform *pl, int32_t n, int64_t b, const int8_t *levels, int32_t atom_level,
                           int32_t dep_mode, int16_t *proc_out, int64_t *start_out, int64_t *finish_out,
                           int32_t *order_out, int64_t *issue_out, or_stats *st) {
    if (n < 1) return OR_ERR_ARG;
    int64_t nb = or_base_count(n);
    int32_t lmax = 0;
    int64_t ntask = 0;
    int32_t *ops = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    if (!ops) return OR_ERR_CAPACITY;
    or_base_ops(n, ops);
    int64_t code_cap = 0;
    for (int64_t t = 0; t < nb; t++) {
        if (levels[t] < 0 || levels[t] > 12) { free(ops); return OR_ERR_ARG; }
        if (levels[t] > lmax) lmax = levels[t];
        /* tasks and code length of a uniform split: 8^l bounds both */
        int64_t c = 1;
        for (int l = 0; l < levels[t]; l++) c *= 8;
        ntask += c;
        code_cap += 2 * c;
    }
    free(ops);
    if (atom_level < 0) atom_level = lmax;
    int8_t *code = (int8_t *)malloc((size_t)code_cap + 1);
    if (!code) return OR_ERR_CAPACITY;
    int64_t len = or_levels_to_code(n, levels, code, code_cap + 1);
    if (len < 0) { free(code); return (int32_t)len; }
    int32_t rc = or_simulate(pl, n, b, code, len, ntask, atom_level, dep_mode, proc_out, start_out, finish_out,
                             order_out, issue_out, st);
    free(code);
    return rc;
}

/* Number of tasks a k-way partition of a task of type op creates, by
 * enumerating the loops of emit(). */
static int64_t part_count(int32_t op, int64_t k) {
    int64_t c = 0;
    if (op == OP_CHOL) {
        for (int64_t p = 0; p < k; p++) {
            c += 1;
            for (int64_t q = p + 1; q < k; q++) c += 1;
            for (int64_t i = p + 1; i < k; i++) {
                for (int64_t q = i + 1; q < k; q++) c += 1;
                c += 1;
            }
        }
    } else if (op == OP_TRSM) {
        for (int64_t p = 0; p < k; p++) {
            c += k;
            for (int64_t i = p + 1; i < k; i++) c += k;
        }
    } else if (op == OP_SYRK) {
        for (int64_t p = 0; p < k; p++)
            for (int64_t i = 0; i < k; i++) c += (k - 1 - i) + 1;
    } else {
        c = k * k * k;
    }
    return c;
}

/* Split code of a one-level partition per base task: base task t is cut
 * with partition parameter p = 1 / factors[t] (factor 1 keeps it); its new
 * tasks are not partitioned again.  Returns the code length or an error. */
int64_t or_factors_to_code(int32_t n, const int8_t *factors, int8_t *code, int64_t cap) {
    int64_t nb = or_base_count(n);
    int32_t *ops = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    if (!ops) return OR_ERR_CAPACITY;
    or_base_ops(n, ops);
    int64_t pos = 0;
    for (int64_t t = 0; t < nb; t++) {
        int32_t f = factors[t];
        if (f < 1 || f > 64) { free(ops); return OR_ERR_ARG; }
        if (pos >= cap) { free(ops); return OR_ERR_CAPACITY; }
        code[pos++] = (int8_t)(f - 1);
        if (f > 1) {
            int64_t kids = part_count(ops[t], f);
            if (pos + kids > cap) { free(ops); return OR_ERR_CAPACITY; }
            for (int64_t q = 0; q < kids; q++) code[pos++] = 0;
        }
    }
    free(ops);
    return pos;
}

static int64_t gcd64(int64_t x, int64_t y) {
    while (y) { int64_t r = x % y; x = y; y = r; }
    return x;
}

/* One candidate of one-level k-way partitions (factors[t] per base task).
 * The atoms are the common refinement of every tiling: side b / L, L the
 * least common multiple of the factors (b must be a multiple of L). */
int32_t or_simulate_factors(const or_platform *pl, int32_t n, int64_t b, const int8_t *factors, int32_t dep_mode,
                            int16_t *proc_out, int64_t *start_out, int64_t *finish_out, int32_t *order_out,
                            int64_t *issue_out, or_stats *st) {
    if (n < 1 || b < 1) return OR_ERR_ARG;
    int64_t nb = or_base_count(n);
    int32_t *ops = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    if (!ops) return OR_ERR_CAPACITY;
    or_base_ops(n, ops);
    int64_t L = 1, ntask = 0;
    for (int64_t t = 0; t < nb; t++) {
        if (factors[t] < 1 || factors[t] > 64) { free(ops); return OR_ERR_ARG; }
        L = L / gcd64(L, factors[t]) * factors[t];
        ntask += factors[t] > 1 ? part_count(ops[t], factors[t]) : 1;
        if (L > b) { free(ops); return OR_ERR_ARG; }
    }
    free(ops);
    if (b % L != 0) return OR_ERR_ARG;
    int64_t cap = ntask + nb;
    int8_t *code = (int8_t *)malloc((size_t)cap);
    if (!code) return OR_ERR_CAPACITY;
    int64_t len = or_factors_to_code(n, factors, code, cap);
    if (len < 0) { free(code); return (int32_t)len; }
    int32_t rc = or_simulate_side(pl, n, b, code, len, ntask, b / L, dep_mode, proc_out, start_out, finish_out,
                                  order_out, issue_out, st);
    free(code);
    return rc;
}

/* Simulate many candidates of the same (n, b), sequentially, one after the
 * other (levels: n_cand x n_base int8). Writes makespans and status. */
int32_t or_simulate_many(const or_platform *pl, int32_t n, int64_t b, const int8_t *levels, int64_t n_cand,
                         int64_t *makespan, int32_t *status, int64_t *tasks) {
    int64_t nb = or_base_count(n);
    for (int64_t c = 0; c < n_cand; c++) {
        or_stats st;
        int32_t rc = or_simulate_levels(pl, n, b, levels + c * nb, -1, 1, NULL, NULL, NULL, NULL, NULL, &st);
        makespan[c] = rc ? -1 : st.makespan;
        status[c] = rc;
        if (tasks) tasks[c] = st.n_tasks;
    }
    return OR_OK;
}
