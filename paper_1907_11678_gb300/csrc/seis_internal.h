// seis_internal.h -- launch parameters shared by the host API and the kernels of libseis.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "seis.h"

namespace seis {

// Device status word bits (read back by seis_device_status).
constexpr unsigned kStatusTimeout = 1u;
constexpr unsigned kStatusOverflow = 2u;   // a staged trace window did not fit (never expected)
constexpr unsigned kStatusBadItem = 4u;    // a batch item with an out-of-range field was skipped

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
    // candidate passes of each tile split over nsplit CTAs (1: no split); with nsplit > 1 the
    // CTAs write their partial argmax to partial[row * nsplit + part] (best S, candidate,
    // stack) and merge_partials_kernel forms the outputs
    int nsplit;
    float4* partial;
};

struct EvalParams {
    const float* traces;
    const int64_t* trace_off;
    const float* h;
    const float* m;
    const int64_t* list_off;
    const int32_t* list;
    const float* m_c;
    const int64_t* out_off;
    const float* dt;
    int64_t nowner;
    int tiles_per_owner;      // ceil(max_rows / 128)
    const float* theta;       // [rows][nparam]
    int nparam;               // 1 (C, CMP) or 3 (A, B, C)
    float* S;                 // [rows] or nullptr
    float* stack;             // [rows] or nullptr
    int32_t* N;               // [rows] or nullptr
    float* grad;              // [rows][3] or nullptr (CRS only)
    unsigned* status;
};

// One refinement step per row (reading c16: projected normalised-gradient ascent).  State:
// theta/S/grad/stack = accepted point, trial_* = the last evaluated trial, step (< 0 once
// the gradient vanished: no further trials).  If `assess`, the trial is accepted when its S is
// not lower, else the step halves.  If `propose`, the next trial is formed.
struct RefineParams {
    int64_t rows;
    float* theta;
    float* S;
    float* grad;
    float* stack;
    float* trial_theta;
    const float* trial_S;
    const float* trial_grad;
    const float* trial_stack;
    float* step;
    float* H;       // [rows][6] inverse curvature estimates (symmetric 3x3)
    float lo[3], hi[3];
    float step0;
    int assess, propose, init;
};

// Launchers (return the cudaError_t of the launch).
cudaError_t launch_search(const SearchParams& p, bool crs, int w, cudaStream_t stream);
cudaError_t launch_merge_partials(const SearchParams& p, bool crs, int64_t rows, cudaStream_t s);
cudaError_t launch_eval(const EvalParams& p, bool crs, bool grad, int w, cudaStream_t s);
cudaError_t launch_refine_update(const RefineParams& r, cudaStream_t s);
int refine_run(const EvalParams& p0, float* theta, const float* lo3, const float* hi3,
               int32_t steps, float step0, int32_t w, float* S_out, float* grad_out,
               float* stack_out, void* workspace, int64_t rows, cudaStream_t s);
int refine_check(const seis_gathers* d, const seis_aperture* ap, const float* theta,
                 const float* lo3, const float* hi3, int32_t steps, float step0, int32_t w,
                 const float* S_out, const float* grad_out, const float* stack_out,
                 const void* workspace, size_t ws_bytes, size_t ws_needed, int64_t rows,
                 EvalParams* p);
int eval_tile_rows();

// Batched search: one persistent launch over items (see seis_batch_semblance).
struct BatchParams {
    const float* traces;
    const int64_t* trace_off;
    const float* h;
    const float* m;
    int64_t ntraces;
    const seis_batch_item* items;
    int64_t nitems;
    int64_t item_begin, item_end;   // the launch serves items [item_begin, item_end)
    const float* poolA;
    const float* poolB;
    const float* poolC;
    int32_t sizeA, sizeB, sizeC;
    int32_t* best_idx;
    float* best_ABC;
    float* best_S;
    float* stack;
    unsigned long long* counter;    // next task (device)
    int64_t* task_off;              // [nitems + 1] first task of each item (device)
    unsigned* status;
    int variant;
};
cudaError_t launch_batch_setup(const BatchParams& p, int64_t out_rows, cudaStream_t s);
cudaError_t launch_batch(const BatchParams& p, int w, int grid, cudaStream_t s);
int batch_variant_of(int search_variant);
int search_variant_count();
const char* search_variant_name(int v);

unsigned* device_status_word();   // this device's status word (module global)

// Error reporting shared by the host entry points (thread-local message).
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* where);

// Autotuner shape buckets: problems in one bucket share the fastest kernel variant.
struct TuneKey {
    int crs, w, cand_bucket, rows_bucket, fold_bucket;
    bool operator<(const TuneKey& o) const {
        if (crs != o.crs) return crs < o.crs;
        if (w != o.w) return w < o.w;
        if (cand_bucket != o.cand_bucket) return cand_bucket < o.cand_bucket;
        if (rows_bucket != o.rows_bucket) return rows_bucket < o.rows_bucket;
        return fold_bucket < o.fold_bucket;
    }
};
TuneKey make_tune_key(bool crs, int w, int ncand, int64_t max_rows, int64_t mean_fold);
void remember_variant(const TuneKey& k, int v);
int lookup_variant(const TuneKey& k, int fallback);
int default_variant();

}  // namespace seis

namespace seis {
struct TuneKey;
int build_cmp_params(const seis_gathers* d, const float* C, int32_t nc, int32_t w, float* S_cube,
                     int32_t* best_idx, float* best_C, float* best_S, float* stack_out,
                     SearchParams* out, TuneKey* key);
int build_crs_params(const seis_gathers* d, const seis_aperture* ap, const float* A, int32_t nA,
                     const float* B, int32_t nB, const float* C, int32_t nC, int32_t w,
                     float* S_cube, int32_t* best_idx, float* best_ABC, float* best_S,
                     float* stack_out, SearchParams* out, TuneKey* key);
}  // namespace seis
