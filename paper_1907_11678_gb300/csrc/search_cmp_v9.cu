// search_cmp_v9.cu -- CMP instantiations of search kernel variant 9.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_cmp_v9(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<false, SearchV9>(p, w, stream);
}

}  // namespace seis
