// search_cmp_v1.cu -- CMP instantiations of search kernel variant 1.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v1(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV1>(p, w, stream);
}

}  // namespace seis
