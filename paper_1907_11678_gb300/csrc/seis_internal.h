// seis_internal.h -- launch parameters shared by the host API and the kernels of libseis.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace seis {

// Device status word bits (read back by seis_device_status).
constexpr unsigned kStatusTimeout = 1u;
constexpr unsigned kStatusOverflow = 2u;   // a staged trace window did not fit (never expected)

// One semblance search launch.  An "owner" is a CMP gather (CMP) or a central CDP (CRS);
// each CTA handles one owner and a tile of 32 consecutive output rows of it.
struct SearchParams {
    const float* traces;
    const int64_t* trace_off;
    const float* h;
    const float* m;            // CRS only
    // owner -> trace list: contiguous gather (list == nullptr) or an aperture list
    const int64_t* list_off;   // [nowner+1]: gather_off (CMP) or nbr_off (CRS)
    const int32_t* list;       // nullptr (CMP) or nbr_trace (CRS)
    const float* m_c;          // CRS central midpoints
    const int64_t* out_off;    // [nowner+1]
    const float* dt;           // [nowner]
    int64_t nowner;
    int tiles_per_owner;       // ceil(max_rows / 32)
    // candidates: cand = (ia*nB + ib)*nC + ic; CMP uses nA = nB = 1 and A = B = nullptr
    const float* A;
    const float* B;
    const float* C;
    int nA, nB, nC, ncand;
    // outputs
    float* S_cube;             // [rows][ncand] or nullptr
    int32_t* best_idx;
    float* best_param;         // [rows] (CMP) or [rows][3] (CRS), or nullptr
    float* best_S;
    float* stack;
    unsigned* status;
    int variant;               // search kernel variant (tile shape / arithmetic form)
};

// Launchers (return the cudaError_t of the launch).
cudaError_t launch_search(const SearchParams& p, bool crs, int w, cudaStream_t stream);
int search_variant_count();
const char* search_variant_name(int v);

unsigned* device_status_word();   // this device's status word (module global)

}  // namespace seis
