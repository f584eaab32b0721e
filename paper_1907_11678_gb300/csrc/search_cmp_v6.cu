// search_cmp_v6.cu -- CMP instantiations of search kernel variant 6.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v6(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV6>(p, w, stream);
}

}  // namespace seis
