// search_cmp_v3.cu -- CMP instantiations of search kernel variant 3.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v3(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV3>(p, w, stream);
}

}  // namespace seis
