// search_crs_v3.cu -- CRS instantiations of search kernel variant 3.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v3(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV3>(p, w, stream);
}

}  // namespace seis
