// search_crs_v2.cu -- CRS instantiations of search kernel variant 2.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v2(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV2>(p, w, stream);
}

}  // namespace seis
