// search_crs_v0.cu -- CRS instantiations of search kernel variant 0.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v0(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV0>(p, w, stream);
}

}  // namespace seis
