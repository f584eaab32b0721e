// search_crs_v4.cu -- CRS instantiations of search kernel variant 4.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v4(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV4>(p, w, stream);
}

}  // namespace seis
