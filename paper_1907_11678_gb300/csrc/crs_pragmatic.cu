// crs_pragmatic.cu -- the CRS operator found by two small searches instead of the dense 3-D
// grid: C from the central CMP's own traces (dm = 0, where the CRS traveltime of Section 2.2
// reduces to the CMP one of Section 2.1), A and B from the zero-offset traces of the aperture
// (h = 0, where the C term vanishes), then S and the stack of the combined operator over the
// full aperture.  The paper searches the dense grid; this decomposition is not in it.
#include <cuda_runtime.h>
#include "seis.h"
#include "seis_internal.h"

namespace seis {

__global__ void pragmatic_consts_kernel(float* zeros2, float* czo, float c_zo) {
    zeros2[0] = 0.f;
    zeros2[1] = 0.f;
    czo[0] = c_zo;
}

// Operator of each row: (A, B) of the zero-offset search, C of the central-CMP search.
__global__ void pragmatic_combine_kernel(int64_t rows, const float* __restrict__ abc_cmp,
                                         const float* __restrict__ abc_zo,
                                         float* __restrict__ abc) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    abc[r * 3 + 0] = abc_zo[r * 3 + 0];
    abc[r * 3 + 1] = abc_zo[r * 3 + 1];
    abc[r * 3 + 2] = abc_cmp[r * 3 + 2];
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace seis

using namespace seis;

extern "C" size_t seis_pragmatic_workspace_size(int64_t rows) {
    if (rows < 0) return 0;
    const size_t r = (size_t)rows;
    // constants; per search: index, operator, S, stack; the trace counts of the final stack
    return 256 + 2 * (align256(r * 4) + align256(r * 12) + align256(r * 4) + align256(r * 4)) +
           align256(r * 4);
}

extern "C" int crs_pragmatic(const seis_gathers* d, const seis_aperture* ap_full,
                             const seis_aperture* ap_cmp, const seis_aperture* ap_zo,
                             const float* A, int32_t nA, const float* B, int32_t nB,
                             const float* C, int32_t nC, float c_zo, int32_t w, float* best_ABC,
                             float* best_S, float* stack_out, void* workspace, size_t ws_bytes,
                             int64_t rows, void* stream) {
    if (!ap_full || !ap_cmp || !ap_zo) return fail(SEIS_EINVAL, "an aperture descriptor is NULL");
    if (ap_cmp->n_central != ap_full->n_central || ap_zo->n_central != ap_full->n_central ||
        ap_cmp->max_rows != ap_full->max_rows || ap_zo->max_rows != ap_full->max_rows)
        return fail(SEIS_EINVAL, "the three apertures must describe the same central CDPs");
    if (!best_ABC || !best_S || !stack_out) return fail(SEIS_EINVAL, "an output array is NULL");
    if (rows < 1) return fail(SEIS_EINVAL, "rows must be >= 1");
    if (!workspace || ws_bytes < seis_pragmatic_workspace_size(rows))
        return fail(SEIS_EINVAL, "workspace of %zu bytes needed", seis_pragmatic_workspace_size(rows));
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return fail(SEIS_EINVAL, "workspace must be 256-byte aligned");
    const size_t r = (size_t)rows;
    char* ws = static_cast<char*>(workspace);
    float* zeros2 = reinterpret_cast<float*>(ws);
    float* czo = zeros2 + 2;
    ws += 256;
    auto take = [&](size_t bytes) { char* p = ws; ws += align256(bytes); return p; };
    int32_t* idx1 = reinterpret_cast<int32_t*>(take(r * 4));
    float* abc1 = reinterpret_cast<float*>(take(r * 12));
    float* S1 = reinterpret_cast<float*>(take(r * 4));
    float* st1 = reinterpret_cast<float*>(take(r * 4));
    int32_t* idx2 = reinterpret_cast<int32_t*>(take(r * 4));
    float* abc2 = reinterpret_cast<float*>(take(r * 12));
    float* S2 = reinterpret_cast<float*>(take(r * 4));
    float* st2 = reinterpret_cast<float*>(take(r * 4));
    int32_t* N = reinterpret_cast<int32_t*>(take(r * 4));
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    pragmatic_consts_kernel<<<1, 1, 0, s>>>(zeros2, czo, c_zo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "crs_pragmatic");
    // C: the central CMP's traces (dm = 0), A = B = 0
    int rc = crs_semblance(d, ap_cmp, zeros2, 1, zeros2 + 1, 1, C, nC, w, nullptr, idx1, abc1, S1,
                           st1, stream);
    if (rc) return rc;
    // A, B: the zero-offset traces of the aperture, C fixed at c_zo (no effect where h = 0)
    rc = crs_semblance(d, ap_zo, A, nA, B, nB, czo, 1, w, nullptr, idx2, abc2, S2, st2, stream);
    if (rc) return rc;
    const int64_t blocks = (rows + 255) / 256;
    pragmatic_combine_kernel<<<(unsigned)blocks, 256, 0, s>>>(rows, abc1, abc2, best_ABC);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "crs_pragmatic combine");
    // S and stack of the combined operator over the full aperture
    return stack(d, ap_full, best_ABC, w, stack_out, best_S, N, stream);
}
