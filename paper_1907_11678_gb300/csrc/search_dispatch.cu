// search_dispatch.cu -- picks the search kernel variant for a launch.
#include "search_kernel.cuh"

namespace seis {

#define SEIS_DECL(name) cudaError_t name(const SearchParams&, int, cudaStream_t);
SEIS_DECL(launch_search_cmp_v0) SEIS_DECL(launch_search_cmp_v1) SEIS_DECL(launch_search_cmp_v2)
SEIS_DECL(launch_search_cmp_v3) SEIS_DECL(launch_search_cmp_v4) SEIS_DECL(launch_search_cmp_v5)
SEIS_DECL(launch_search_crs_v0) SEIS_DECL(launch_search_crs_v1) SEIS_DECL(launch_search_crs_v2)
SEIS_DECL(launch_search_crs_v3) SEIS_DECL(launch_search_crs_v4) SEIS_DECL(launch_search_crs_v5)
SEIS_DECL(launch_search_cmp_v6) SEIS_DECL(launch_search_cmp_v7) SEIS_DECL(launch_search_cmp_v8)
SEIS_DECL(launch_search_cmp_v9) SEIS_DECL(launch_search_crs_v6) SEIS_DECL(launch_search_crs_v7)
SEIS_DECL(launch_search_crs_v8) SEIS_DECL(launch_search_crs_v9)
SEIS_DECL(launch_search_cmp_v10) SEIS_DECL(launch_search_crs_v10)
#undef SEIS_DECL

int search_variant_count() { return kSearchVariants; }

const char* search_variant_name(int v) {
    switch (v) {
        case 0: return "7 warps x 4 candidates, packed f32x2";
        case 1: return "7 warps x 4 candidates, scalar";
        case 2: return "11 warps x 2 candidates, hybrid (scalar difference, packed interpolation)";
        case 3: return "11 warps x 2 candidates, scalar";
        case 4: return "15 warps x 2 candidates, packed f32x2";
        case 5: return "15 warps x 2 candidates, scalar";
        case 6: return "11 warps x 2 candidates, hybrid (scalar interpolation, packed sums)";
        case 7: return "15 warps x 2 candidates, hybrid (scalar interpolation, packed sums)";
        case 8: return "7 warps x 4 candidates, hybrid (scalar difference, packed interpolation)";
        case 9: return "7 warps x 4 candidates, hybrid (scalar interpolation, packed sums)";
        case 10: return "12 warps x 2 candidates, packed f32x2 (three per warp scheduler)";
        default: return "";
    }
}

cudaError_t launch_search(const SearchParams& p, bool crs, int w, cudaStream_t stream) {
    typedef cudaError_t (*fn_t)(const SearchParams&, int, cudaStream_t);
    static const fn_t cmp[kSearchVariants] = {
        launch_search_cmp_v0, launch_search_cmp_v1, launch_search_cmp_v2, launch_search_cmp_v3,
        launch_search_cmp_v4, launch_search_cmp_v5, launch_search_cmp_v6, launch_search_cmp_v7,
        launch_search_cmp_v8, launch_search_cmp_v9, launch_search_cmp_v10};
    static const fn_t crsf[kSearchVariants] = {
        launch_search_crs_v0, launch_search_crs_v1, launch_search_crs_v2, launch_search_crs_v3,
        launch_search_crs_v4, launch_search_crs_v5, launch_search_crs_v6, launch_search_crs_v7,
        launch_search_crs_v8, launch_search_crs_v9, launch_search_crs_v10};
    if (p.variant < 0 || p.variant >= kSearchVariants) return cudaErrorInvalidValue;
    return (crs ? crsf : cmp)[p.variant](p, w, stream);
}

}  // namespace seis
