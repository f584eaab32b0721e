// batch_api.cu -- C ABI of the batched search (seis_batch_semblance): item validation and
// the task table (a one-CTA scan on the device), then one persistent launch or one launch
// per item.
#include <cuda_runtime.h>
#include <vector>
#include "seis.h"
#include "seis_internal.h"
#include "batch_scratch.h"
#include "seis_dev.cuh"

namespace seis {

cudaError_t launch_batch_v0(const BatchParams&, int, int, cudaStream_t);
cudaError_t launch_batch_v1(const BatchParams&, int, int, cudaStream_t);
cudaError_t launch_batch_v3(const BatchParams&, int, int, cudaStream_t);
cudaError_t launch_batch_v4(const BatchParams&, int, int, cudaStream_t);
cudaError_t launch_batch_v9(const BatchParams&, int, int, cudaStream_t);
cudaError_t launch_batch_v10(const BatchParams&, int, int, cudaStream_t);

// The batch kernel is instantiated for six of the search variants (its per-task state
// costs registers, so most hybrid shapes are left out); any other choice maps to variant 3.
static const int kBatchVariants[] = {0, 1, 3, 4, 9, 10};
int batch_variant_of(int v) {
    for (int b : kBatchVariants)
        if (b == v) return v;
    return 3;
}

cudaError_t launch_batch(const BatchParams& p, int w, int grid, cudaStream_t s) {
    switch (batch_variant_of(p.variant)) {
        case 0: return launch_batch_v0(p, w, grid, s);
        case 1: return launch_batch_v1(p, w, grid, s);
        case 4: return launch_batch_v4(p, w, grid, s);
        case 9: return launch_batch_v9(p, w, grid, s);
        case 10: return launch_batch_v10(p, w, grid, s);
        default: return launch_batch_v3(p, w, grid, s);
    }
}

// Tuning key of the batched search: one bucket per window length.
static TuneKey batch_key(int w) { return TuneKey{2, w, 0, 0, 0}; }

// One CTA: validate every item (an invalid one gets no tasks and sets the status bit),
// prefix-sum the tiles of 32 rows into task_off, zero the work counter.
__global__ void batch_setup_kernel(const BatchParams P, int64_t out_rows) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) { carry = 0; *P.counter = 0ull; P.task_off[0] = 0; }
    __syncthreads();
    for (int64_t i0 = 0; i0 < P.nitems; i0 += blockDim.x) {
        const int64_t i = i0 + tid;
        int64_t tiles = 0;
        if (i < P.nitems) {
            const seis_batch_item it = P.items[i];
            const bool crs = it.kind == 1;
            const int64_t nA = crs ? it.nA : 1, nB = crs ? it.nB : 1;
            bool ok = (it.kind == 0 || it.kind == 1) && it.trace_begin >= 0 &&
                      it.trace_begin <= it.trace_end && it.trace_end <= P.ntraces &&
                      it.rows >= 0 && it.rows < (1 << 24) && it.out_begin >= 0 &&
                      it.out_begin + it.rows <= out_rows && it.nC >= 1 && it.c_off >= 0 &&
                      (int64_t)it.c_off + it.nC <= P.sizeC && it.dt > 0.f &&
                      nA * nB * (int64_t)it.nC <= ((int64_t)1 << 30);
            if (crs)
                ok = ok && P.m && it.nA >= 1 && it.nB >= 1 && it.a_off >= 0 && it.b_off >= 0 &&
                     (int64_t)it.a_off + it.nA <= P.sizeA && (int64_t)it.b_off + it.nB <= P.sizeB;
            if (ok) tiles = (it.rows + 31) / 32;
            else record_status(P.status, kStatusBadItem);
        }
        int64_t x = tiles;                                   // inclusive scan in the block
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int64_t before = carry;
        for (int w2 = 0; w2 < warp; ++w2) before += wsum[w2];
        if (i < P.nitems) P.task_off[i + 1] = before + x;
        __syncthreads();
        if (tid == 0) {
            int64_t tot = 0;
            for (int w2 = 0; w2 < nw; ++w2) tot += wsum[w2];
            carry += tot;
        }
        __syncthreads();
    }
}

cudaError_t launch_batch_setup(const BatchParams& p, int64_t out_rows, cudaStream_t s) {
    batch_setup_kernel<<<1, 1024, 0, s>>>(p, out_rows);
    return cudaGetLastError();
}

}  // namespace seis

using namespace seis;

extern "C" size_t seis_batch_workspace_size(int64_t nitems) {
    return batch_workspace_bytes(nitems);
}

namespace seis {

// Checks the arguments of seis_batch_semblance and fills the launch parameters.
static int batch_prepare(const seis_gathers* d, const seis_batch_item* items, int64_t nitems,
                         const float* poolA, int32_t sizeA, const float* poolB, int32_t sizeB,
                         const float* poolC, int32_t sizeC, int32_t w, int32_t mode,
                         int32_t* best_idx, float* best_ABC, float* best_S, float* stack_out,
                         int64_t out_rows, void* workspace, size_t ws_bytes, BatchParams* out) {
    if (!d || !d->traces || !d->trace_off || !d->half_offset)
        return fail(SEIS_EINVAL, "gathers descriptor or its trace arrays are NULL");
    if ((reinterpret_cast<uintptr_t>(d->traces) & 3u) != 0)
        return fail(SEIS_EINVAL, "traces must be 4-byte aligned");
    if (d->ntraces < 0) return fail(SEIS_EINVAL, "ntraces must be >= 0");
    if (d->max_trace_samples < 0 || d->max_trace_samples > SEIS_MAX_TRACE_SAMPLES)
        return fail(SEIS_EINVAL, "max_trace_samples %d outside [0, %d]", d->max_trace_samples,
                    SEIS_MAX_TRACE_SAMPLES);
    if (w < 1 || (w % 2) == 0 || w > SEIS_MAX_W)
        return fail(SEIS_EINVAL, "window w = %d must be odd and in [1, %d]", w, SEIS_MAX_W);
    if (!items || nitems < 1) return fail(SEIS_EINVAL, "items must be non-NULL, nitems >= 1");
    if (!poolC || sizeC < 1 || sizeA < 0 || sizeB < 0)
        return fail(SEIS_EINVAL, "candidate pools: poolC needed, sizes >= 0");
    if (mode != 0 && mode != 1) return fail(SEIS_EINVAL, "mode must be 0 or 1");
    if (!best_idx || !best_S || !stack_out || out_rows < 0)
        return fail(SEIS_EINVAL, "an output array is NULL");
    if (!workspace || ws_bytes < seis_batch_workspace_size(nitems))
        return fail(SEIS_EINVAL, "workspace of %zu bytes needed", seis_batch_workspace_size(nitems));
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return fail(SEIS_EINVAL, "workspace must be 256-byte aligned");
    BatchParams p{};
    p.traces = d->traces;
    p.trace_off = d->trace_off;
    p.h = d->half_offset;
    p.m = d->midpoint;
    p.ntraces = d->ntraces;
    p.items = items;
    p.nitems = nitems;
    p.poolA = poolA;
    p.poolB = poolB;
    p.poolC = poolC;
    p.sizeA = poolA ? sizeA : 0;
    p.sizeB = poolB ? sizeB : 0;
    p.sizeC = sizeC;
    p.best_idx = best_idx;
    p.best_ABC = best_ABC;
    p.best_S = best_S;
    p.stack = stack_out;
    p.counter = static_cast<unsigned long long*>(workspace);
    p.task_off = reinterpret_cast<int64_t*>(static_cast<char*>(workspace) + 256);
    p.status = device_status_word();
    p.variant = lookup_variant(batch_key(w), default_variant());
    *out = p;
    return SEIS_OK;
}

// Task table, then the persistent launch (mode 0) or one launch per item (mode 1).
static int batch_run(BatchParams p, int32_t w, int32_t mode, int64_t out_rows, cudaStream_t s) {
    cudaError_t e = launch_batch_setup(p, out_rows, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch setup");
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "batch");
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "batch");
    if (mode == 0) {
        p.item_begin = 0;
        p.item_end = p.nitems;
        if ((e = launch_batch(p, w, 2 * sms, s)) != cudaSuccess) return cuda_fail(e, "batch launch");
        return SEIS_OK;
    }
    // one launch per item: the task table is read back to size each launch
    std::vector<int64_t> off((size_t)p.nitems + 1);
    e = cudaMemcpyAsync(off.data(), p.task_off, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "batch per-item");
    for (int64_t i = 0; i < p.nitems; ++i) {
        const int64_t tasks = off[i + 1] - off[i];
        if (tasks <= 0) continue;
        p.item_begin = i;
        p.item_end = i + 1;
        if ((e = cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), s)) != cudaSuccess)
            return cuda_fail(e, "batch per-item");
        const int grid = (int)(tasks < 2 * sms ? tasks : 2 * sms);
        if ((e = launch_batch(p, w, grid, s)) != cudaSuccess) return cuda_fail(e, "batch launch");
    }
    return SEIS_OK;
}

}  // namespace seis

extern "C" int seis_batch_semblance(const seis_gathers* d, const seis_batch_item* items,
                                    int64_t nitems, const float* poolA, int32_t sizeA,
                                    const float* poolB, int32_t sizeB, const float* poolC,
                                    int32_t sizeC, int32_t w, int32_t mode, int32_t* best_idx,
                                    float* best_ABC, float* best_S, float* stack_out,
                                    int64_t out_rows, void* workspace, size_t ws_bytes,
                                    void* stream) {
    BatchParams p;
    int rc = batch_prepare(d, items, nitems, poolA, sizeA, poolB, sizeB, poolC, sizeC, w, mode,
                           best_idx, best_ABC, best_S, stack_out, out_rows, workspace, ws_bytes,
                           &p);
    if (rc) return rc;
    return batch_run(p, w, mode, out_rows, static_cast<cudaStream_t>(stream));
}

extern "C" int seis_autotune_batch(const seis_gathers* d, const seis_batch_item* items,
                                   int64_t nitems, const float* poolA, int32_t sizeA,
                                   const float* poolB, int32_t sizeB, const float* poolC,
                                   int32_t sizeC, int32_t w, int32_t* best_idx, float* best_ABC,
                                   float* best_S, float* stack_out, int64_t out_rows,
                                   void* workspace, size_t ws_bytes, int32_t reps,
                                   int32_t* chosen, float* ms_out, void* stream) {
    BatchParams p;
    int rc = batch_prepare(d, items, nitems, poolA, sizeA, poolB, sizeB, poolC, sizeC, w, 0,
                           best_idx, best_ABC, best_S, stack_out, out_rows, workspace, ws_bytes,
                           &p);
    if (rc) return rc;
    if (reps < 1) reps = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ms_out)
        for (int v = 0; v < search_variant_count(); ++v) ms_out[v] = -1.f;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(e, "batch autotune"); }
    int best = -1;
    float best_ms = 0.f;
    for (int v : kBatchVariants) {
        p.variant = v;
        float ms = 0.f;
        rc = batch_run(p, w, 0, out_rows, s);                  // untimed
        if (!rc && (e = cudaEventRecord(e0, s)) != cudaSuccess) rc = cuda_fail(e, "batch autotune");
        for (int r = 0; r < reps && !rc; ++r) rc = batch_run(p, w, 0, out_rows, s);
        if (!rc && (e = cudaEventRecord(e1, s)) != cudaSuccess) rc = cuda_fail(e, "batch autotune");
        if (!rc && (e = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(e, "batch autotune");
        if (!rc && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
            rc = cuda_fail(e, "batch autotune");
        if (rc) break;
        ms /= (float)reps;
        if (ms_out) ms_out[v] = ms;
        if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    remember_variant(batch_key(w), best);
    if (chosen) *chosen = best;
    return SEIS_OK;
}
