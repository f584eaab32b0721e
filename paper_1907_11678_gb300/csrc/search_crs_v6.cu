// search_crs_v6.cu -- CRS instantiations of search kernel variant 6.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v6(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV6>(p, w, stream);
}

}  // namespace seis
