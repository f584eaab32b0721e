// search_crs_v8.cu -- CRS instantiations of search kernel variant 8.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v8(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV8>(p, w, stream);
}

}  // namespace seis
