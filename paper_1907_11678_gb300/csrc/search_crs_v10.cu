// search_crs_v10.cu -- CRS instantiations of search kernel variant 10.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v10(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV10>(p, w, stream);
}

}  // namespace seis
