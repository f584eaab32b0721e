// batch_v10.cu -- batch kernel instantiations of search kernel variant 10.
#include "batch_kernel.cuh"

namespace seis {

cudaError_t launch_batch_v10(const BatchParams& p, int w, int grid, cudaStream_t s) {
    return launch_batch_cfg<SearchV10>(p, w, grid, s);
}

}  // namespace seis
