// eval_api.cu -- C ABI of the per-row operator evaluation: stack, crs_semblance_grad and
// crs_refine (declared in include/seis.h).
#include <cuda_runtime.h>
#include "seis.h"
#include "seis_internal.h"
#include "eval_pair.h"

namespace seis {

static int build_eval(const seis_gathers* d, const seis_aperture* ap, const float* theta,
                      int32_t w, EvalParams* out, int64_t* rows) {
    if (!d) return fail(SEIS_EINVAL, "gathers descriptor is NULL");
    if (!d->traces || !d->trace_off || !d->half_offset || !d->gather_off || !d->out_off || !d->dt)
        return fail(SEIS_EINVAL, "a required gathers array is NULL");
    if ((reinterpret_cast<uintptr_t>(d->traces) & 3u) != 0)
        return fail(SEIS_EINVAL, "traces must be 4-byte aligned");
    if (d->ngathers < 1) return fail(SEIS_EINVAL, "ngathers must be >= 1");
    if (d->max_trace_samples < 0 || d->max_trace_samples > SEIS_MAX_TRACE_SAMPLES)
        return fail(SEIS_EINVAL, "max_trace_samples %d outside [0, %d]", d->max_trace_samples,
                    SEIS_MAX_TRACE_SAMPLES);
    if (w < 1 || (w % 2) == 0 || w > SEIS_MAX_W)
        return fail(SEIS_EINVAL, "window w = %d must be odd and in [1, %d]", w, SEIS_MAX_W);
    if (!theta) return fail(SEIS_EINVAL, "operator array is NULL");
    EvalParams p{};
    p.traces = d->traces;
    p.trace_off = d->trace_off;
    p.h = d->half_offset;
    p.theta = theta;
    p.status = device_status_word();
    if (ap) {
        if (!d->midpoint) return fail(SEIS_EINVAL, "midpoint array is NULL");
        if (!ap->nbr_off || !ap->nbr_trace || !ap->m_c || !ap->out_off || !ap->dt)
            return fail(SEIS_EINVAL, "an aperture array is NULL");
        if (ap->n_central < 1 || ap->max_rows < 1)
            return fail(SEIS_EINVAL, "aperture needs n_central >= 1 and max_rows >= 1");
        p.m = d->midpoint;
        p.list_off = ap->nbr_off;
        p.list = ap->nbr_trace;
        p.m_c = ap->m_c;
        p.out_off = ap->out_off;
        p.dt = ap->dt;
        p.nowner = ap->n_central;
        p.tiles_per_owner = (ap->max_rows + eval_tile_rows() - 1) / eval_tile_rows();
        p.nparam = 3;
    } else {
        if (d->max_rows < 1) return fail(SEIS_EINVAL, "max_rows must be >= 1");
        p.list_off = d->gather_off;
        p.out_off = d->out_off;
        p.dt = d->dt;
        p.nowner = d->ngathers;
        p.tiles_per_owner = (d->max_rows + eval_tile_rows() - 1) / eval_tile_rows();
        p.nparam = 1;
    }
    *out = p;
    *rows = 0;
    return SEIS_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace seis

using namespace seis;

extern "C" int stack(const seis_gathers* d, const seis_aperture* ap, const float* params,
                     int32_t w, float* stack_out, float* S_out, int32_t* N_out, void* stream) {
    EvalParams p;
    int64_t rows;
    int rc = build_eval(d, ap, params, w, &p, &rows);
    if (rc) return rc;
    if (!stack_out) return fail(SEIS_EINVAL, "stack_out is NULL");
    p.stack = stack_out;
    p.S = S_out;
    p.N = N_out;
    cudaError_t e = launch_eval(p, ap != nullptr, false, w, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stack launch");
    return SEIS_OK;
}

extern "C" int crs_semblance_grad(const seis_gathers* d, const seis_aperture* ap,
                                  const float* ABC, int32_t w, float* S_out, float* grad_out,
                                  float* stack_out, void* stream) {
    if (!ap) return fail(SEIS_EINVAL, "aperture descriptor is NULL");
    EvalParams p;
    int64_t rows;
    int rc = build_eval(d, ap, ABC, w, &p, &rows);
    if (rc) return rc;
    if (!S_out || !grad_out) return fail(SEIS_EINVAL, "S_out and grad_out are required");
    p.S = S_out;
    p.grad = grad_out;
    p.stack = stack_out;
    cudaError_t e = launch_eval(p, true, true, w, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "crs_semblance_grad launch");
    return SEIS_OK;
}

extern "C" size_t seis_refine_workspace_size(int64_t rows) {
    if (rows < 0) return 0;
    const size_t r = (size_t)rows;
    return align256(r * 3 * 4) + align256(r * 4) + align256(r * 3 * 4) + align256(r * 4) +
           align256(r * 4) + align256(r * 6 * 4);
}

namespace seis {

// The refinement loop of crs_refine on caller-checked arguments: theta [rows][3] in/out,
// S, grad, stack outputs, ws of seis_refine_workspace_size(rows) bytes (256-aligned).  With
// `pair`, the state holds two starts of the same rows ([2][rows][...]) and each evaluation
// is one paired launch (eval_pair.cu); the update kernel runs over all 2 rows states.
static int refine_loop(const EvalParams& p0, float* theta, const float* lo3, const float* hi3,
                       int32_t steps, float step0, int32_t w, float* S_out, float* grad_out,
                       float* stack_out, void* workspace, int64_t rows, bool pair,
                       cudaStream_t s) {
    const int64_t nstate = pair ? 2 * rows : rows;
    char* ws = static_cast<char*>(workspace);
    const size_t r = (size_t)nstate;
    float* trial_theta = reinterpret_cast<float*>(ws);
    ws += align256(r * 3 * 4);
    float* trial_S = reinterpret_cast<float*>(ws);
    ws += align256(r * 4);
    float* trial_grad = reinterpret_cast<float*>(ws);
    ws += align256(r * 3 * 4);
    float* trial_stack = reinterpret_cast<float*>(ws);
    ws += align256(r * 4);
    float* step = reinterpret_cast<float*>(ws);
    ws += align256(r * 4);
    float* Hinv = reinterpret_cast<float*>(ws);

    RefineParams u{};
    u.rows = nstate;
    u.theta = theta;
    u.S = S_out;
    u.grad = grad_out;
    u.stack = stack_out;
    u.trial_theta = trial_theta;
    u.trial_S = trial_S;
    u.trial_grad = trial_grad;
    u.trial_stack = trial_stack;
    u.step = step;
    u.H = Hinv;
    for (int a = 0; a < 3; ++a) { u.lo[a] = lo3[a]; u.hi[a] = hi3[a]; }
    u.step0 = step0;

    // one evaluation of the operators th into the trial outputs
    auto evaluate = [&](const float* th) -> cudaError_t {
        EvalParams p = p0;
        p.theta = th;
        p.S = trial_S;
        p.grad = trial_grad;
        p.stack = trial_stack;
        if (!pair) return launch_eval(p, true, true, w, s);
        EvalPairParams q{};
        q.p = p;
        q.theta2 = th + rows * 3;
        q.S2 = trial_S + rows;
        q.grad2 = trial_grad + rows * 3;
        q.stack2 = trial_stack + rows;
        return launch_eval_pair(q, w, s);
    };
    cudaError_t e = evaluate(theta);                   // the starting operators
    if (e != cudaSuccess) return cuda_fail(e, "crs_refine eval");
    u.init = 1;
    u.assess = 0;
    u.propose = steps > 0;
    if ((e = launch_refine_update(u, s)) != cudaSuccess) return cuda_fail(e, "crs_refine update");
    u.init = 0;
    for (int it = 0; it < steps; ++it) {
        if ((e = evaluate(trial_theta)) != cudaSuccess) return cuda_fail(e, "crs_refine eval");
        u.assess = 1;
        u.propose = it + 1 < steps;
        if ((e = launch_refine_update(u, s)) != cudaSuccess) return cuda_fail(e, "crs_refine update");
    }
    return SEIS_OK;
}

int refine_run(const EvalParams& p0, float* theta, const float* lo3, const float* hi3,
               int32_t steps, float step0, int32_t w, float* S_out, float* grad_out,
               float* stack_out, void* workspace, int64_t rows, cudaStream_t s) {
    return refine_loop(p0, theta, lo3, hi3, steps, step0, w, S_out, grad_out, stack_out,
                       workspace, rows, false, s);
}

int refine_run_pair(const EvalParams& p0, float* theta, const float* lo3, const float* hi3,
                    int32_t steps, float step0, int32_t w, float* S_out, float* grad_out,
                    float* stack_out, void* workspace, int64_t rows, cudaStream_t s) {
    return refine_loop(p0, theta, lo3, hi3, steps, step0, w, S_out, grad_out, stack_out,
                       workspace, rows, true, s);
}

// Argument checks shared by crs_refine and crs_refine_multi.
int refine_check(const seis_gathers* d, const seis_aperture* ap, const float* theta,
                 const float* lo3, const float* hi3, int32_t steps, float step0, int32_t w,
                 const float* S_out, const float* grad_out, const float* stack_out,
                 const void* workspace, size_t ws_bytes, size_t ws_needed, int64_t rows,
                 EvalParams* p) {
    if (!ap) return fail(SEIS_EINVAL, "aperture descriptor is NULL");
    int64_t dummy;
    int rc = build_eval(d, ap, theta, w, p, &dummy);
    if (rc) return rc;
    if (!lo3 || !hi3) return fail(SEIS_EINVAL, "lo3 / hi3 are NULL");
    for (int a = 0; a < 3; ++a)
        if (!(hi3[a] > lo3[a])) return fail(SEIS_EINVAL, "hi3[%d] must exceed lo3[%d]", a, a);
    if (steps < 0 || !(step0 > 0.f)) return fail(SEIS_EINVAL, "steps >= 0 and step0 > 0 needed");
    if (!S_out || !grad_out || !stack_out) return fail(SEIS_EINVAL, "an output array is NULL");
    if (rows < 1) return fail(SEIS_EINVAL, "rows must be >= 1");
    if (!workspace || ws_bytes < ws_needed)
        return fail(SEIS_EINVAL, "workspace of %zu bytes needed", ws_needed);
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return fail(SEIS_EINVAL, "workspace must be 256-byte aligned");
    return SEIS_OK;
}

}  // namespace seis

extern "C" int crs_refine(const seis_gathers* d, const seis_aperture* ap, float* ABC_inout,
                          const float* lo3, const float* hi3, int32_t steps, float step0,
                          int32_t w, float* S_out, float* grad_out, float* stack_out,
                          void* workspace, size_t ws_bytes, int64_t rows, void* stream) {
    EvalParams p;
    int rc = refine_check(d, ap, ABC_inout, lo3, hi3, steps, step0, w, S_out, grad_out,
                          stack_out, workspace, ws_bytes, seis_refine_workspace_size(rows), rows,
                          &p);
    if (rc) return rc;
    return refine_run(p, ABC_inout, lo3, hi3, steps, step0, w, S_out, grad_out, stack_out,
                      workspace, rows, static_cast<cudaStream_t>(stream));
}
