// search_cmp_v5.cu -- CMP instantiations of search kernel variant 5.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v5(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV5>(p, w, stream);
}

}  // namespace seis
