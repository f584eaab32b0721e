// search_split.cu -- the semblance search of problems too small to fill the GPU
// (cmp_semblance_ws, crs_semblance_ws, seis_search_workspace_size; declared in seis.h).
//
// A search grid has one CTA per (owner, tile of 32 rows), so a few owners leave most SMs
// idle.  Here each tile's candidate passes are split over nsplit CTAs, each writing the
// argmax of its own candidates (best S, candidate, stack) to a caller workspace, and a merge
// kernel takes, per row, the best S over the parts (the split kernel is instantiated for the
// default tile shape only, so the plain search compiles as without it).  Every candidate's
// sums are formed as in
// the unsplit search (same traces, same order), the parts cover increasing candidate ranges
// and the merge keeps the earlier part on ties, so the outputs are bit-identical to
// cmp_semblance / crs_semblance.
#include <algorithm>
#include <climits>
#include <cuda_runtime.h>
#include "seis.h"
#include "seis_internal.h"
#include "search_kernel.cuh"

namespace seis {

template <bool CRS>
__global__ void merge_partials_kernel(const SearchParams P, int64_t rows) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float4* q = P.partial + r * P.nsplit;
    float bs = -1.f, bt = 0.f;
    int bc = 0;
    for (int k = 0; k < P.nsplit; ++k) {           // parts in candidate order
        const float4 v = q[k];
        if (v.x > bs) { bs = v.x; bc = __float_as_int(v.y); bt = v.z; }
    }
    P.best_idx[r] = bc;
    P.best_S[r] = bs;
    P.stack[r] = bt;
    if (P.best_param) {
        float a, b, cc;
        decode_candidate<CRS>(P, bc, a, b, cc);
        if (CRS) {
            P.best_param[r * 3 + 0] = a;
            P.best_param[r * 3 + 1] = b;
            P.best_param[r * 3 + 2] = cc;
        } else {
            P.best_param[r] = cc;
        }
    }
}

cudaError_t launch_merge_partials(const SearchParams& p, bool crs, int64_t rows, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const int64_t blocks = (rows + 255) / 256;
    if (blocks > INT_MAX) return cudaErrorInvalidValue;
    if (crs) merge_partials_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(p, rows);
    else merge_partials_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(p, rows);
    return cudaGetLastError();
}

// SMs of the current device (cached per device).
static int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}

// Parts per tile.  The CTAs of a launch run in waves of `slots` (2 resident search CTAs per
// SM); a grid of g CTAs keeps the GPU busy for the fraction (g / slots) / ceil(g / slots) of
// its waves.  Take the smallest part count whose grid reaches 90 % (else the best one up to
// about 4 waves), with at least one candidate pass per part (no variant takes more than 32
// candidates per pass); 1 when the tiles alone do.
static int split_count(int64_t n_owner, int32_t max_rows, int64_t ncand) {
    const int64_t grid = n_owner * (((int64_t)max_rows + 31) / 32);
    const int64_t slots = 2 * (int64_t)sm_count();
    if (grid <= 0 || slots <= 0) return 1;
    auto fill = [&](int64_t k) {
        const int64_t ctas = grid * k;
        return (double)ctas / (double)(((ctas + slots - 1) / slots) * slots);
    };
    if (fill(1) >= 0.9) return 1;
    const int64_t cap = std::min<int64_t>((ncand + 31) / 32,
                                          std::max<int64_t>(2, (4 * slots + grid - 1) / grid));
    int64_t best = 1;
    for (int64_t k = 2; k <= cap; ++k) {
        if (fill(k) >= 0.9) return (int)k;
        if (fill(k) > fill(best) + 1e-9) best = k;
    }
    return (int)best;
}

static int run_split(SearchParams& p, bool crs, int w, int64_t rows, void* workspace,
                     size_t ws_bytes, cudaStream_t s, const char* who) {
    const int k = split_count(p.nowner, p.tiles_per_owner * 32, p.ncand);
    cudaError_t e;
    if (k > 1) {
        const size_t need = (size_t)rows * k * sizeof(float4);
        if (!workspace || ws_bytes < need)
            return fail(SEIS_EINVAL, "%s: workspace of %zu bytes needed", who, need);
        if ((reinterpret_cast<uintptr_t>(workspace) & 15u) != 0)
            return fail(SEIS_EINVAL, "%s: workspace must be 16-byte aligned", who);
        p.nsplit = k;
        p.partial = static_cast<float4*>(workspace);
        // the split kernel is built for the default tile shape (variant 4: 15 warps x 2
        // candidates, packed f32x2), the fastest on every measured workload
        e = crs ? launch_search_cfg<true, SearchV4, true>(p, w, s)
                : launch_search_cfg<false, SearchV4, true>(p, w, s);
        if (e != cudaSuccess) return cuda_fail(e, who);
        if ((e = launch_merge_partials(p, crs, rows, s)) != cudaSuccess) return cuda_fail(e, who);
        return SEIS_OK;
    }
    if ((e = launch_search(p, crs, w, s)) != cudaSuccess) return cuda_fail(e, who);
    return SEIS_OK;
}

}  // namespace seis

using namespace seis;

extern "C" size_t seis_search_workspace_size(int64_t n_owner, int32_t max_rows, int64_t rows,
                                             int64_t ncand) {
    if (n_owner < 1 || max_rows < 1 || rows < 0 || ncand < 1) return 0;
    const int k = split_count(n_owner, max_rows, ncand);
    return k > 1 ? (size_t)rows * k * sizeof(float4) : 0;
}

extern "C" int cmp_semblance_ws(const seis_gathers* d, const float* C, int32_t nc, int32_t w,
                                float* S_cube, int32_t* best_idx, float* best_C, float* best_S,
                                float* stack_out, void* workspace, size_t ws_bytes, int64_t rows,
                                void* stream) {
    SearchParams p;
    TuneKey key;
    int rc = build_cmp_params(d, C, nc, w, S_cube, best_idx, best_C, best_S, stack_out, &p, &key);
    if (rc) return rc;
    if (rows < 0) return fail(SEIS_EINVAL, "rows must be >= 0");
    return run_split(p, false, w, rows, workspace, ws_bytes, static_cast<cudaStream_t>(stream),
                     "cmp_semblance_ws");
}

extern "C" int crs_semblance_ws(const seis_gathers* d, const seis_aperture* ap, const float* A,
                                int32_t nA, const float* B, int32_t nB, const float* C, int32_t nC,
                                int32_t w, float* S_cube, int32_t* best_idx, float* best_ABC,
                                float* best_S, float* stack_out, void* workspace, size_t ws_bytes,
                                int64_t rows, void* stream) {
    SearchParams p;
    TuneKey key;
    int rc = build_crs_params(d, ap, A, nA, B, nB, C, nC, w, S_cube, best_idx, best_ABC, best_S,
                              stack_out, &p, &key);
    if (rc) return rc;
    if (rows < 0) return fail(SEIS_EINVAL, "rows must be >= 0");
    return run_split(p, true, w, rows, workspace, ws_bytes, static_cast<cudaStream_t>(stream),
                     "crs_semblance_ws");
}
