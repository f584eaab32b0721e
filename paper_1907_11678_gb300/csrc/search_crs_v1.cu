// search_crs_v1.cu -- CRS instantiations of search kernel variant 1.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v1(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV1>(p, w, stream);
}

}  // namespace seis
