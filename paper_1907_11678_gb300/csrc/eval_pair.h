// eval_pair.h -- the paired evaluation of two CRS operators per output row (eval_pair.cu) and
// the refinement loop that drives it two starts at a time.
#pragma once
#include "seis_internal.h"

namespace seis {

// p describes the rows, the first operator set (p.theta) and its outputs (p.S, p.stack,
// p.grad); the second set and its outputs follow.  CRS only, always with the adjoint.
struct EvalPairParams {
    EvalParams p;
    const float* theta2;
    float* S2;
    float* stack2;
    float* grad2;
};

cudaError_t launch_eval_pair(const EvalPairParams& q, int w, cudaStream_t s);

// crs_refine's loop for two starts at once: theta [2][rows][3] in/out, S_out, stack_out
// [2][rows], grad_out [2][rows][3], workspace of seis_refine_workspace_size(2 * rows) bytes.
// Every output equals two separate refine_run calls bit for bit.
int refine_run_pair(const EvalParams& p0, float* theta, const float* lo3, const float* hi3,
                    int32_t steps, float step0, int32_t w, float* S_out, float* grad_out,
                    float* stack_out, void* workspace, int64_t rows, cudaStream_t s);

}  // namespace seis
