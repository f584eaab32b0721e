// search_cmp_v4.cu -- CMP instantiations of search kernel variant 4.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v4(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV4>(p, w, stream);
}

}  // namespace seis
