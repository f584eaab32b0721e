// batch_v0.cu -- batch kernel instantiations of search kernel variant 0.
#include "batch_kernel.cuh"

namespace seis {

cudaError_t launch_batch_v0(const BatchParams& p, int w, int grid, cudaStream_t s) {
    return launch_batch_cfg<SearchV0>(p, w, grid, s);
}

}  // namespace seis
