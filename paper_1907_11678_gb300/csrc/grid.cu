// grid.cu -- the candidate grids of the semblance search (seis_velocity_grid,
// seis_linear_grid; declared in include/seis.h).
//
// Section 3.2 generates the NMO velocity array from its upper and lower bounds: here nc
// velocities linearly spaced over [vmin, vmax], both bounds included, each turned into the
// stacking parameter C = 4/v^2 of the hyperbola t^2 = t0^2 + C h^2 in half-offset h.  The
// CRS axes A, B and C are plain linear grids.  Every value is formed in FP64 with explicitly
// rounded operations (no contraction into fused multiply-adds) and rounded once to FP32.
#include <cmath>
#include <cuda_runtime.h>
#include "seis.h"
#include "seis_internal.h"

namespace seis {

// lo + (hi - lo) * i / (n - 1) in FP64, lo itself when n == 1.
__device__ __forceinline__ double grid_point(double lo, double hi, int i, int n) {
    if (n == 1) return lo;
    const double frac = __ddiv_rn(__dmul_rn(__dsub_rn(hi, lo), (double)i), (double)(n - 1));
    return __dadd_rn(lo, frac);
}

__global__ void velocity_grid_kernel(double vmin, double vmax, int nc, float* C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double v = grid_point(vmin, vmax, i, nc);
    C[i] = (float)__ddiv_rn(4.0, __dmul_rn(v, v));
}

__global__ void linear_grid_kernel(double lo, double hi, int n, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = (float)grid_point(lo, hi, i, n);
}

}  // namespace seis

using namespace seis;

extern "C" int seis_velocity_grid(double vmin, double vmax, int32_t nc, float* C_out,
                                  void* stream) {
    if (!C_out) return fail(SEIS_EINVAL, "C_out is NULL");
    if (nc < 1) return fail(SEIS_EINVAL, "nc must be >= 1, got %d", nc);
    if (!(std::isfinite(vmin) && std::isfinite(vmax) && vmin > 0.0 && vmax > 0.0))
        return fail(SEIS_EINVAL, "velocity bounds must be finite and positive");
    velocity_grid_kernel<<<(nc + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        vmin, vmax, nc, C_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SEIS_OK : cuda_fail(e, "seis_velocity_grid launch");
}

extern "C" int seis_linear_grid(double lo, double hi, int32_t n, float* out, void* stream) {
    if (!out) return fail(SEIS_EINVAL, "out is NULL");
    if (n < 1) return fail(SEIS_EINVAL, "n must be >= 1, got %d", n);
    if (!(std::isfinite(lo) && std::isfinite(hi))) return fail(SEIS_EINVAL, "bounds must be finite");
    linear_grid_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(lo, hi, n,
                                                                                      out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SEIS_OK : cuda_fail(e, "seis_linear_grid launch");
}
