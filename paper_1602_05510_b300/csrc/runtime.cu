// Runtime services around the kernels: CUDA-graph capture and replay of any
// sequence of asynchronous library calls, and the launch-shape autotuner of
// the simulator with an on-disk cache.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "hesp_internal.h"

struct hesp_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

int hesp_graph_begin(void *stream) {
    if (!stream) return HESP_ERR_ARG;  // the legacy default stream cannot be captured
    return cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeRelaxed) == cudaSuccess ? HESP_OK
                                                                                                     : HESP_ERR_CUDA;
}

int hesp_graph_end(void *stream, hesp_graph **out) {
    if (!stream || !out) return HESP_ERR_ARG;
    *out = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture((cudaStream_t)stream, &g) != cudaSuccess || !g) return HESP_ERR_CUDA;
    cudaGraphExec_t e = nullptr;
    if (cudaGraphInstantiate(&e, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return HESP_ERR_CUDA;
    }
    hesp_graph *h = (hesp_graph *)calloc(1, sizeof(hesp_graph));
    if (!h) {
        cudaGraphExecDestroy(e);
        cudaGraphDestroy(g);
        return HESP_ERR_CAPACITY;
    }
    h->graph = g;
    h->exec = e;
    *out = h;
    return HESP_OK;
}

int hesp_graph_launch(const hesp_graph *g, void *stream) {
    if (!g) return HESP_ERR_ARG;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? HESP_OK : HESP_ERR_CUDA;
}

void hesp_graph_destroy(hesp_graph *g) {
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    free(g);
}

int hesp_platform_set_tuning(hesp_platform *p, int32_t ctas_per_sm, int32_t bitmap_place) {
    if (!p || ctas_per_sm < 0 || ctas_per_sm > 64 || bitmap_place < 0 || bitmap_place > 2) return HESP_ERR_ARG;
    p->tune_ctas_per_sm = ctas_per_sm;
    p->tune_bitmap = bitmap_place;
    return HESP_OK;
}

int hesp_platform_get_tuning(const hesp_platform *p, int32_t *ctas_per_sm, int32_t *bitmap_place) {
    if (!p || !ctas_per_sm || !bitmap_place) return HESP_ERR_ARG;
    *ctas_per_sm = p->tune_ctas_per_sm;
    *bitmap_place = p->tune_bitmap;
    return HESP_OK;
}

static void tune_key(const hesp_platform *p, int32_t max_tiles, int32_t max_level, int64_t task_cap, char *key,
                     size_t n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof prop);
    cudaGetDeviceProperties(&prop, dev);
    char name[128];
    snprintf(name, sizeof name, "%s", prop.name);
    for (char *c = name; *c; ++c)
        if (*c == ' ' || *c == '|') *c = '_';
    snprintf(key, n, "%s|sm%d|t%d|l%d|task%lld|m%d|p%d", name, prop.multiProcessorCount, max_tiles, max_level,
             (long long)task_cap, p->n_mem, p->n_procs);
}

static std::mutex g_cache_mu;

static int cache_lookup(const char *path, const char *key, int *ctas, int *bm) {
    FILE *f = fopen(path, "r");
    if (!f) return 0;
    char line[512], k[400];
    int c = 0, b = 0, found = 0;
    while (fgets(line, sizeof line, f))
        if (sscanf(line, "%399s %d %d", k, &c, &b) == 3 && strcmp(k, key) == 0) {
            *ctas = c;
            *bm = b;
            found = 1;
        }
    fclose(f);
    return found;
}

// Time the simulation of a sample batch under every launch shape (1..max CTAs
// of 8 candidate warps per SM, release bitmap in shared or global memory),
// keep the fastest in the platform handle, and remember it in cache_path
// (nullable) keyed by GPU, problem bounds and platform shape.  Synchronous.
// ms_out (nullable, 8 entries) receives each shape's time, -1 where skipped.
int hesp_sim_autotune(hesp_platform *p, const hesp_cand *cands_dev, const int8_t *levels_dev, int64_t n_sample,
                      int32_t max_tiles, int32_t max_level, int64_t task_cap, int64_t *makespan_dev,
                      int32_t *status_dev, void *ws, size_t ws_bytes, const char *cache_path, int32_t *best_ctas,
                      int32_t *best_bitmap, float *ms_out, void *stream) {
    if (!p || !cands_dev || !levels_dev || n_sample < 1 || !makespan_dev || !status_dev || !ws) return HESP_ERR_ARG;
    char key[400];
    tune_key(p, max_tiles, max_level, task_cap, key, sizeof key);
    if (ms_out)
        for (int i = 0; i < 8; ++i) ms_out[i] = -1.f;
    if (cache_path) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        int c = 0, b = 0;
        if (cache_lookup(cache_path, key, &c, &b)) {
            p->tune_ctas_per_sm = c;
            p->tune_bitmap = b;
            if (best_ctas) *best_ctas = c;
            if (best_bitmap) *best_bitmap = b;
            return HESP_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HESP_ERR_CUDA;
    const int32_t old_c = p->tune_ctas_per_sm, old_b = p->tune_bitmap;
    float best = 1e30f;
    int bc = 0, bb = 0, rc = HESP_OK;
    for (int bmp = 1; bmp <= 2 && !rc; ++bmp)
        for (int ctas = 1; ctas <= 4 && !rc; ++ctas) {
            p->tune_ctas_per_sm = ctas;
            p->tune_bitmap = bmp;
            // warm-up, then one timed run
            rc = hesp_simulate_batch(p, cands_dev, levels_dev, n_sample, max_tiles, max_level, task_cap, makespan_dev,
                                     status_dev, nullptr, nullptr, nullptr, nullptr, nullptr, ws, ws_bytes, stream);
            if (rc) break;
            cudaEventRecord(e0, st);
            rc = hesp_simulate_batch(p, cands_dev, levels_dev, n_sample, max_tiles, max_level, task_cap, makespan_dev,
                                     status_dev, nullptr, nullptr, nullptr, nullptr, nullptr, ws, ws_bytes, stream);
            cudaEventRecord(e1, st);
            if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = rc ? rc : HESP_ERR_CUDA;
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms_out) ms_out[(bmp - 1) * 4 + ctas - 1] = ms;
            if (ms < best) {
                best = ms;
                bc = ctas;
                bb = bmp;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        p->tune_ctas_per_sm = old_c;
        p->tune_bitmap = old_b;
        return rc;
    }
    p->tune_ctas_per_sm = bc;
    p->tune_bitmap = bb;
    if (best_ctas) *best_ctas = bc;
    if (best_bitmap) *best_bitmap = bb;
    if (cache_path) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s %d %d\n", key, bc, bb);
            fclose(f);
        }
    }
    return HESP_OK;
}

}  // extern "C"
