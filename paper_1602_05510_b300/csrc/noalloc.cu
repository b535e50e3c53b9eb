// hesp_simulate_batch_noalloc: the batched simulation without a caller-
// supplied workspace and without any device allocation.
//
// Some callers cannot allocate device memory at the moment they want to
// simulate: code that runs under a memory manager which owns the whole device
// budget and forbids allocations outside it, plugin hosts that hand a library
// only the buffers of its inputs and outputs, or loops with a hard latency
// bound where a cudaMalloc (which may synchronise the device) is not allowed.
// For them the per-candidate arenas live in one fixed array in the library's
// own device memory, sized HESP_NOALLOC_SCRATCH_BYTES; every GPU that loads
// the library holds that array until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "hesp_internal.h"

namespace {

// The scratch array.  In host code its name is only a host-side stand-in: the
// device address is obtained with cudaGetSymbolAddress per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HESP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
int scratch_for_current_device(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HESP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (err != cudaSuccess || !ptr) return HESP_ERR_CUDA;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return HESP_OK;
}

}  // namespace

extern "C" int hesp_simulate_batch_noalloc(const hesp_platform *p, const hesp_cand *cands_dev,
                                           const int8_t *levels_dev, int64_t n_cand, int32_t max_tiles,
                                           int32_t max_level, int64_t *makespan_dev, int32_t *status_dev,
                                           int64_t *ntasks_dev, const int64_t *sched_offsets_dev, int16_t *proc_dev,
                                           int64_t *start_dev, int64_t *finish_dev, void *stream) {
    if (!p || n_cand < 0) return HESP_ERR_ARG;
    if (max_tiles < 1 || max_tiles > HESP_MAX_TILES || max_level < 0 || max_level > HESP_MAX_LEVEL)
        return HESP_ERR_UNSUPPORTED;
    // One candidate arena (plus the work-counter header) must fit the array.
    const hesp::Arena ar = hesp::make_arena(max_tiles, max_level, p->n_mem, 0, hesp::arena_room_of(p));
    if (hesp::kWsHeaderBytes + ar.slot_bytes > (int64_t)HESP_NOALLOC_SCRATCH_BYTES) return HESP_ERR_CAPACITY;
    if (n_cand == 0) return HESP_OK;
    void *scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    // The work counter at the head of the array is reset by every launch and
    // every arena is fully re-initialised per candidate, so nothing left by an
    // earlier call is read.
    return hesp_simulate_batch(p, cands_dev, levels_dev, n_cand, max_tiles, max_level, 0, makespan_dev, status_dev,
                               ntasks_dev, sched_offsets_dev, proc_dev, start_dev, finish_dev, scratch,
                               (size_t)HESP_NOALLOC_SCRATCH_BYTES, stream);
}
