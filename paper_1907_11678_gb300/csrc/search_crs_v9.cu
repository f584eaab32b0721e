// search_crs_v9.cu -- CRS instantiations of search kernel variant 9.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs_v9(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_cfg<true, SearchV9>(p, w, stream);
}

}  // namespace seis
