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

// Starts at the local maxima of a row's coarse cube: one warp per row.  The warp first
// marks, in a bitmask in shared memory, every candidate whose (S, -index) exceeds that of
// each of its grid neighbours (ia, ib, ic each within +-1); then k selection passes take
// the best entries in the order (local maxima first, then S descending, then index
// ascending), as top_starts_kernel does without the first key.
constexpr int kLmWarps = 4;                      // rows (warps) per block
__global__ void local_max_starts_kernel(const float* __restrict__ S, int64_t rows, int nA,
                                        int nB, int nC, const float* __restrict__ A,
                                        const float* __restrict__ B,
                                        const float* __restrict__ C, int k,
                                        float* __restrict__ out) {
    extern __shared__ unsigned lm_bits[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * kLmWarps + warp;
    if (row >= rows) return;                       // uniform over the warp
    const int ncand = nA * nB * nC;
    const int nwords = (ncand + 31) / 32;
    unsigned* bits = lm_bits + warp * nwords;
    const float* Sr = S + row * (int64_t)ncand;
    for (int w0 = 0; w0 < nwords; ++w0) {          // 32 candidates per round, one per lane
        const int c = w0 * 32 + lane;
        bool lmax = false;
        if (c < ncand) {
            const int ia = c / (nB * nC), rem = c - ia * nB * nC;
            const int ib = rem / nC, ic = rem - ib * nC;
            const float v = Sr[c];
            lmax = true;
            for (int da = -1; da <= 1 && lmax; ++da) {
                const int a = ia + da;
                if (a < 0 || a >= nA) continue;
                for (int db = -1; db <= 1 && lmax; ++db) {
                    const int b = ib + db;
                    if (b < 0 || b >= nB) continue;
                    for (int dc = -1; dc <= 1; ++dc) {
                        const int cc = ic + dc;
                        if (cc < 0 || cc >= nC || (da == 0 && db == 0 && dc == 0)) continue;
                        const int n = (a * nB + b) * nC + cc;
                        const float u = Sr[n];
                        if (u > v || (u == v && n < c)) { lmax = false; break; }
                    }
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, lmax);
        if (lane == 0) bits[w0] = m;
    }
    __syncwarp();
    // selection: key (group, S, index) with group 0 for local maxima, ordered (group asc,
    // S desc, index asc); pass j takes the smallest key after pass j-1's pick
    int lastG = -1, lastI = -1;
    float lastS = FLT_MAX;
    for (int j = 0; j < k; ++j) {
        int bg = 2, bi = INT_MAX;
        float bs = -FLT_MAX;
        for (int c = lane; c < ncand; c += 32) {
            const int g = ((bits[c >> 5] >> (c & 31)) & 1u) ? 0 : 1;
            const float v = Sr[c];
            const bool after = g > lastG || (g == lastG && (v < lastS || (v == lastS && c > lastI)));
            const bool better = g < bg || (g == bg && (v > bs || (v == bs && c < bi)));
            if (after && better) { bg = g; bs = v; bi = c; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const int og = __shfl_xor_sync(0xffffffffu, bg, o);
            const float os = __shfl_xor_sync(0xffffffffu, bs, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (og < bg || (og == bg && (os > bs || (os == bs && oi < bi)))) {
                bg = og; bs = os; bi = oi;
            }
        }
        if (bi == INT_MAX) bi = 0;                   // unreachable for k <= ncand
        lastG = bg;
        lastS = bs;
        lastI = bi;
        if (lane == 0) {
            const int ia = bi / (nB * nC), rem = bi - ia * nB * nC;
            const int ib = rem / nC, ic = rem - ib * nC;
            float* o = out + ((int64_t)j * rows + row) * 3;
            o[0] = A[ia];
            o[1] = B[ib];
            o[2] = C[ic];
        }
    }
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
extern "C" int crs_local_max_starts(const float* S_cube, int64_t rows, const float* A,
                                    int32_t nA, const float* B, int32_t nB, const float* C,
                                    int32_t nC, int32_t nstart, float* ABC_starts, void* stream) {
    if (!S_cube || !A || !B || !C || !ABC_starts) return fail(SEIS_EINVAL, "an array is NULL");
    if (rows < 1) return fail(SEIS_EINVAL, "rows must be >= 1");
    if (nA < 1 || nB < 1 || nC < 1) return fail(SEIS_EINVAL, "empty candidate axis");
    const int64_t ncand = (int64_t)nA * nB * nC;
    if (ncand > SEIS_LOCAL_MAX_CANDIDATES)
        return fail(SEIS_EUNSUPPORTED, "%lld candidates, at most %d", (long long)ncand,
                    SEIS_LOCAL_MAX_CANDIDATES);
    if (nstart < 1 || nstart > ncand)
        return fail(SEIS_EINVAL, "nstart = %d outside [1, %lld]", nstart, (long long)ncand);
    const int64_t blocks = (rows + kLmWarps - 1) / kLmWarps;
    if (blocks > INT_MAX) return fail(SEIS_EINVAL, "too many rows");
    // one bit per candidate and row: at most 16 KB per block, within the default limit
    const size_t smem = (size_t)kLmWarps * ((ncand + 31) / 32) * sizeof(unsigned);
    local_max_starts_kernel<<<(unsigned)blocks, 32 * kLmWarps, smem,
                              static_cast<cudaStream_t>(stream)>>>(
        S_cube, rows, nA, nB, nC, A, B, C, nstart, ABC_starts);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "crs_local_max_starts launch");
    return SEIS_OK;
}

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
