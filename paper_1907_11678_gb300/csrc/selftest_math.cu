// selftest_math.cu -- measures the relative error of the fast square root and reciprocal the
// search kernels use for the traveltime (seis_selftest_fast_math, declared in seis.h).
#include <cuda_runtime.h>
#include "seis.h"
#include "seis_internal.h"
#include "seis_dev.cuh"

namespace seis {

// Every float x in [1, 4) -- 2^24 consecutive bit patterns, all mantissas under both
// exponent parities -- against FP64: the largest |sqrt_fast(x) - sqrt(x)| / sqrt(x) and
// |rcp_fast(x) - 1/x| * x, as float bit patterns (non-negative, so integer order is float
// order) reduced with atomicMax.
__global__ void fast_math_error_kernel(unsigned* out) {
    float es = 0.f, er = 0.f;
    const unsigned first = 0x3F800000u;            // 1.0f
    const unsigned count = 1u << 24;               // up to 4.0f (exclusive)
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += gridDim.x * blockDim.x) {
        const float x = __uint_as_float(first + i);
        const double xd = (double)x;
        const double sd = sqrt(xd);
        es = fmaxf(es, (float)(fabs((double)sqrt_fast(x) - sd) / sd));
        er = fmaxf(er, (float)(fabs((double)rcp_fast(x) - 1.0 / xd) * xd));
    }
    for (int o = 16; o > 0; o >>= 1) {
        es = fmaxf(es, __shfl_xor_sync(0xffffffffu, es, o));
        er = fmaxf(er, __shfl_xor_sync(0xffffffffu, er, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, __float_as_uint(es));
        atomicMax(out + 1, __float_as_uint(er));
    }
}

}  // namespace seis

using namespace seis;

extern "C" int seis_selftest_fast_math(float* max_rel_err, void* stream) {
    if (!max_rel_err) return fail(SEIS_EINVAL, "max_rel_err is NULL");
    if ((reinterpret_cast<uintptr_t>(max_rel_err) & 3u) != 0)
        return fail(SEIS_EINVAL, "max_rel_err must be 4-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(max_rel_err, 0, 2 * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "seis_selftest_fast_math");
    fast_math_error_kernel<<<1024, 256, 0, s>>>(reinterpret_cast<unsigned*>(max_rel_err));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "seis_selftest_fast_math launch");
    return SEIS_OK;
}
