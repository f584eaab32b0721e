// batch_noalloc.cu -- an allocation-free entry point to the batched search.
//
// seis_batch_semblance needs a small device scratch area (a work counter and the task
// table) that the caller allocates.  Some callers cannot allocate device memory where they
// call this library: a processing service that runs under a fixed device-memory budget
// set at start-up, a plug-in whose host application owns every allocation, or a latency-
// bound loop that cannot afford cudaMalloc (which may synchronise the device).  For them,
// seis_batch_semblance_noalloc keeps that scratch in a file-scope device array instead.
//
// The array lives in this library's module on every GPU that loads the library and stays
// resident until the process exits.  Its size bounds the number of items per call.  All
// calls share it: each call rebuilds the task table and resets the counter before the
// search kernel reads them, and calls whose work overlaps on the GPU (different streams,
// other host threads) race on it.
#include <cuda_runtime.h>
#include "seis.h"
#include "seis_internal.h"
#include "batch_scratch.h"

namespace seis {

// [0, 256): the work counter; [256, ...): the task table (SEIS_NOALLOC_MAX_ITEMS + 1 int64,
// rounded up to 256 bytes) -- exactly what seis_batch_workspace_size(SEIS_NOALLOC_MAX_ITEMS)
// asks of a caller workspace, so a call with the maximum item count passes its check.
static constexpr size_t kNoallocBytes = batch_workspace_bytes(SEIS_NOALLOC_MAX_ITEMS);
static_assert(kNoallocBytes == 256 + 8 * ((size_t)SEIS_NOALLOC_MAX_ITEMS + 1) + 248,
              "the array holds the counter and the 256-byte-rounded task table of the maximum "
              "item count");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The array's device address, looked up once per device with that device current.  It stays
// valid for the life of the device's primary context (a cudaDeviceReset ends it).
static void* g_noalloc_addr[64] = {};

static int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "seis_batch_semblance_noalloc");
    if (dev < 0 || dev >= 64) return fail(SEIS_EUNSUPPORTED, "device index %d above 63", dev);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "seis_batch_semblance_noalloc scratch address");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SEIS_OK;
}

}  // namespace seis

using namespace seis;

extern "C" int seis_batch_semblance_noalloc(const seis_gathers* d, const seis_batch_item* items,
                                            int64_t nitems, const float* poolA, int32_t sizeA,
                                            const float* poolB, int32_t sizeB,
                                            const float* poolC, int32_t sizeC, int32_t w,
                                            int32_t* best_idx, float* best_ABC, float* best_S,
                                            float* stack_out, int64_t out_rows, void* stream) {
    if (nitems > SEIS_NOALLOC_MAX_ITEMS)
        return fail(SEIS_EINVAL, "seis_batch_semblance_noalloc takes at most %d items, got %lld",
                    SEIS_NOALLOC_MAX_ITEMS, (long long)nitems);
    void* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    // Same checks and launches as the persistent mode of seis_batch_semblance, with the
    // library's own scratch array as the workspace.
    return seis_batch_semblance(d, items, nitems, poolA, sizeA, poolB, sizeB, poolC, sizeC, w, 0,
                                best_idx, best_ABC, best_S, stack_out, out_rows, scratch,
                                kNoallocBytes, stream);
}
