// search_cmp_v7.cu -- CMP instantiations of search kernel variant 7.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v7(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV7>(p, w, stream);
}

}  // namespace seis
