// refine_multi.cu -- multi-start refinement of the CRS operators: the best coarse
// candidates of each row as starting points (crs_top_starts) and one refinement per start
// with the best result kept per row (crs_refine_multi).  Neither has a counterpart in the
// paper, whose CRS search is the dense grid of Section 2.2.
#include <cfloat>
#include <climits>
#include <cuda_runtime.h>
#include "seis.h"
#include "seis_internal.h"
#include "seis_dev.cuh"
#include "eval_pair.h"

namespace seis {

// One warp per row: the k largest entries of the row's S cube in the order (S descending,
// candidate index ascending), decoded to (A, B, C) with cand = (ia*nB + ib)*nC + ic.
// Pass j takes the best entry that comes after pass j-1's pick in that order.
__global__ void top_starts_kernel(const float* __restrict__ S, int64_t rows, int ncand,
                                  const float* __restrict__ A, int nA,
                                  const float* __restrict__ B, int nB,
                                  const float* __restrict__ C, int nC, int k,
                                  float* __restrict__ out) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;                       // uniform over the warp
    const float* Sr = S + row * (int64_t)ncand;
    float lastS = FLT_MAX;
    int lastI = -1;
    int first = 0;
    for (int j = 0; j < k; ++j) {
        float bs = -FLT_MAX;
        int bi = INT_MAX;
        for (int c = lane; c < ncand; c += 32) {
            const float v = Sr[c];
            const bool after = (v < lastS) || (v == lastS && c > lastI);
            const bool better = (v > bs) || (v == bs && c < bi);
            if (after && better) { bs = v; bi = c; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, bs, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (os > bs || (os == bs && oi < bi)) { bs = os; bi = oi; }
        }
        if (bi == INT_MAX) bi = first;             // fewer orderable entries than k (NaN)
        if (j == 0) first = bi;
        lastS = bs;
        lastI = bi;
        if (lane == 0) {
            const int nbc = nB * nC;
            const int ia = bi / nbc, rem = bi - ia * nbc;
            const int ib = rem / nC, ic = rem - ib * nC;
            float* o = out + ((int64_t)j * rows + row) * 3;
            o[0] = A[ia];
            o[1] = B[ib];
            o[2] = C[ic];
        }
    }
    (void)nA;
}

// Keep, per row, the refinement with the highest S (the earlier start on ties).
__global__ void keep_best_kernel(int64_t rows, int start, const float* __restrict__ th,
                                 const float* __restrict__ S, const float* __restrict__ g,
                                 const float* __restrict__ st, float* __restrict__ th_best,
                                 float* __restrict__ S_best, float* __restrict__ g_best,
                                 float* __restrict__ st_best) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    if (start == 0 || S[r] > S_best[r]) {
        S_best[r] = S[r];
        st_best[r] = st[r];
        for (int a = 0; a < 3; ++a) {
            th_best[r * 3 + a] = th[r * 3 + a];
            g_best[r * 3 + a] = g[r * 3 + a];
        }
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace seis

using namespace seis;

extern "C" int crs_top_starts(const float* S_cube, int64_t rows, const float* A, int32_t nA,
                              const float* B, int32_t nB, const float* C, int32_t nC,
                              int32_t nstart, float* ABC_starts, void* stream) {
    if (!S_cube || !A || !B || !C || !ABC_starts) return fail(SEIS_EINVAL, "an array is NULL");
    if (rows < 1) return fail(SEIS_EINVAL, "rows must be >= 1");
    if (nA < 1 || nB < 1 || nC < 1) return fail(SEIS_EINVAL, "empty candidate axis");
    const int64_t ncand = (int64_t)nA * nB * nC;
    if (ncand > INT_MAX) return fail(SEIS_EINVAL, "too many candidates");
    if (nstart < 1 || nstart > ncand)
        return fail(SEIS_EINVAL, "nstart = %d outside [1, %lld]", nstart, (long long)ncand);
    const int64_t blocks = (rows * 32 + 255) / 256;
    if (blocks > INT_MAX) return fail(SEIS_EINVAL, "too many rows");
    top_starts_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        S_cube, rows, (int)ncand, A, nA, B, nB, C, nC, nstart, ABC_starts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "crs_top_starts launch");
    return SEIS_OK;
}

// Starts are refined two at a time (the paired evaluation kernel), so the refinement state
// and the per-start results hold two starts of every row.
extern "C" size_t seis_refine_multi_workspace_size(int64_t rows) {
    if (rows < 0) return 0;
    const size_t r2 = 2 * (size_t)rows;
    return seis_refine_workspace_size(2 * rows) + align256(r2 * 3 * 4) + align256(r2 * 4) +
           align256(r2 * 3 * 4) + align256(r2 * 4);
}

extern "C" int crs_refine_multi(const seis_gathers* d, const seis_aperture* ap,
                                const float* ABC_starts, int32_t nstart, const float* lo3,
                                const float* hi3, int32_t steps, float step0, int32_t w,
                                float* ABC_out, float* S_out, float* grad_out, float* stack_out,
                                void* workspace, size_t ws_bytes, int64_t rows, void* stream) {
    if (!ABC_starts || !ABC_out) return fail(SEIS_EINVAL, "ABC_starts / ABC_out are NULL");
    if (nstart < 1) return fail(SEIS_EINVAL, "nstart must be >= 1");
    EvalParams p;
    int rc = refine_check(d, ap, ABC_starts, lo3, hi3, steps, step0, w, S_out, grad_out,
                          stack_out, workspace, ws_bytes, seis_refine_multi_workspace_size(rows),
                          rows, &p);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t r = (size_t)rows, r2 = 2 * r;
    char* ws = static_cast<char*>(workspace);
    void* ws_refine = ws;
    ws += seis_refine_workspace_size(2 * rows);
    float* th = reinterpret_cast<float*>(ws);           // [2][rows][3]: starts k and k+1
    ws += align256(r2 * 3 * 4);
    float* S = reinterpret_cast<float*>(ws);            // [2][rows]
    ws += align256(r2 * 4);
    float* g = reinterpret_cast<float*>(ws);
    ws += align256(r2 * 3 * 4);
    float* st = reinterpret_cast<float*>(ws);
    const int64_t blocks = (rows + 255) / 256;
    if (blocks > INT_MAX) return fail(SEIS_EINVAL, "too many rows");
    for (int k = 0; k < nstart; k += 2) {
        const int npair = (k + 1 < nstart) ? 2 : 1;      // an odd last start runs alone
        cudaError_t e = cudaMemcpyAsync(th, ABC_starts + (size_t)k * r * 3,
                                        npair * r * 3 * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "crs_refine_multi start copy");
        rc = npair == 2 ? refine_run_pair(p, th, lo3, hi3, steps, step0, w, S, g, st, ws_refine,
                                          rows, s)
                        : refine_run(p, th, lo3, hi3, steps, step0, w, S, g, st, ws_refine, rows,
                                     s);
        if (rc) return rc;
        for (int q = 0; q < npair; ++q) {                 // start k before start k+1 (ties)
            keep_best_kernel<<<(unsigned)blocks, 256, 0, s>>>(
                rows, k + q, th + q * r * 3, S + q * r, g + q * r * 3, st + q * r, ABC_out,
                S_out, grad_out, stack_out);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "crs_refine_multi keep");
        }
    }
    return SEIS_OK;
}
