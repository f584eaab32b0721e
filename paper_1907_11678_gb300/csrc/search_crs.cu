// search_crs.cu -- CRS instantiations of the semblance search kernel.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs(const SearchParams& p, int w, cudaStream_t stream) {
    return launch_search_dispatch<true>(p, w, stream);
}

}  // namespace seis
