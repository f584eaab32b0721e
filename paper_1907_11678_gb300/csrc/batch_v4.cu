// batch_v4.cu -- batch kernel instantiations of search kernel variant 4.
#include "batch_kernel.cuh"

namespace seis {

cudaError_t launch_batch_v4(const BatchParams& p, int w, int grid, cudaStream_t s) {
    return launch_batch_cfg<SearchV4>(p, w, grid, s);
}

}  // namespace seis
