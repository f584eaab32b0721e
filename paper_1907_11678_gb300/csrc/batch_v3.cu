// batch_v3.cu -- batch kernel instantiations of search kernel variant 3.
#include "batch_kernel.cuh"

namespace seis {

cudaError_t launch_batch_v3(const BatchParams& p, int w, int grid, cudaStream_t s) {
    return launch_batch_cfg<SearchV3>(p, w, grid, s);
}

}  // namespace seis
