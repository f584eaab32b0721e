// search_cmp_v10.cu -- CMP instantiations of search kernel variant 10.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v10(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV10>(p, w, stream);
}

}  // namespace seis
