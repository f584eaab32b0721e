// search_crs_v7.cu -- CRS instantiations of search kernel variant 7.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v7(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV7>(p, w, stream);
}

}  // namespace seis
