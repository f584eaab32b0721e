// search_cmp_v0.cu -- CMP instantiations of search kernel variant 0.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v0(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV0>(p, w, stream);
}

}  // namespace seis
