// batch_v9.cu -- batch kernel instantiations of search kernel variant 9.
#include "batch_kernel.cuh"

namespace seis {

cudaError_t launch_batch_v9(const BatchParams& p, int w, int grid, cudaStream_t s) {
    return launch_batch_cfg<SearchV9>(p, w, grid, s);
}

}  // namespace seis
