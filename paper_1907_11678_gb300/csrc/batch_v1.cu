// batch_v1.cu -- batch kernel instantiations of search kernel variant 1.
#include "batch_kernel.cuh"

namespace seis {

cudaError_t launch_batch_v1(const BatchParams& p, int w, int grid, cudaStream_t s) {
    return launch_batch_cfg<SearchV1>(p, w, grid, s);
}

}  // namespace seis
