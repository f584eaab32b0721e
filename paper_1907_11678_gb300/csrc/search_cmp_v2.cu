// search_cmp_v2.cu -- CMP instantiations of search kernel variant 2.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v2(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV2>(p, w, stream);
}

}  // namespace seis
