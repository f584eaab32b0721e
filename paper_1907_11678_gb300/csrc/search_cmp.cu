// search_cmp.cu -- CMP instantiations of the semblance search kernel and the dispatcher.
#include "search_kernel.cuh"

namespace seis {

cudaError_t launch_search_crs(const SearchParams& p, int w, cudaStream_t stream);

cudaError_t launch_search(const SearchParams& p, bool crs, int w, cudaStream_t stream) {
    if (crs) return launch_search_crs(p, w, stream);
    return launch_search_dispatch<false>(p, w, stream);
}

}  // namespace seis
