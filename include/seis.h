/*
 * seis.h -- C ABI of libseis: the semblance search of the CMP and CRS stacking methods
 * (arXiv:1907.11678, "Massively Scaling Seismic Processing on Sunway TaihuLight
 * Supercomputer") on one NVIDIA GB300 GPU (sm_103a).
 *
 * Conventions shared by every entry point
 *   - Every array pointer is a DEVICE pointer owned by the caller, unless its comment
 *     says "host".  The library never frees or keeps caller memory.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream).  Outputs are valid once the stream reaches
 *     that point.  Entry points marked SYNCHRONOUS wait on the stream themselves.
 *   - Layouts are row-major.  Traces are stored back to back: trace i is
 *     traces[trace_off[i] .. trace_off[i+1]) (FP32), sample s at time s*dt.
 *   - An "output row" is one output time sample t0 = n*dt of one gather (CMP) or one
 *     central CDP (CRS); rows of owner g are out_off[g] .. out_off[g+1]-1.
 *   - Return codes: SEIS_OK (0) or a negative error; nothing aborts, throws or prints.
 *     seis_last_error() returns a thread-local message for the last failure.
 *   - The offset and index arrays (trace_off, gather_off, out_off, nbr_off, nbr_trace)
 *     live in device memory and are not validated: they must be non-decreasing, index
 *     inside the arrays they describe, and agree with the host-side counts passed beside
 *     them (ngathers, ntraces, max_rows, n_central, and the `rows` of crs_refine,
 *     crs_refine_multi and crs_pragmatic).  The kernels index through them, so offsets
 *     that break these rules can make a kernel read or write outside the caller's
 *     arrays.  Host-side sizes and pointers are checked on every call, and the batch
 *     entry point range-checks each item on the device (see seis_batch_item).
 *   - A device wait that does not finish within about 2 s (a bulk copy that never
 *     lands) makes the kernel record SEIS_ETIMEOUT in the device status word and
 *     return; seis_device_status() reports and clears it.
 *
 * Method readings fixed by this library (the paper is silent on them):
 *   - window j = -hw..hw with hw = w/2 (w odd); one interpolation fraction per trace;
 *   - a trace takes part for a (t0, candidate) only if samples k-hw .. k+hw+1 all lie in
 *     the trace (k = floor of the traveltime in samples) and the traveltime is real
 *     (CRS also needs t0 + A dm >= 0); N counts the traces that take part;
 *   - S = sum_j (sum_i v_ij)^2 / (N sum_j sum_i v_ij^2), 0 when N = 0 or the energy is 0;
 *   - ties of the argmax go to the lowest candidate index;
 *   - stack = (sum_i sum_j v_ij) / (N w) at the picked candidate, 0 when N = 0.
 */
#ifndef SEIS_H
#define SEIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEIS_OK            0
#define SEIS_EINVAL       (-1)   /* an argument is invalid (message in seis_last_error) */
#define SEIS_ECUDA        (-2)   /* a CUDA runtime call failed */
#define SEIS_ETIMEOUT     (-3)   /* a bounded device wait gave up */
#define SEIS_EUNSUPPORTED (-4)   /* valid but outside what this build supports */

/* Largest trace length (samples) the staged kernels accept, and the supported windows. */
#define SEIS_MAX_TRACE_SAMPLES 12280
#define SEIS_MAX_W 15            /* w must be odd, 1 <= w <= SEIS_MAX_W */

/* A set of gathers (Section 3.2: ncdps CDPs of up to `fold` traces of ns samples, traces
 * of a CDP stored contiguously). */
typedef struct seis_gathers {
    const float*   traces;       /* [trace_off[ntraces]] samples, 4-byte aligned           */
    const int64_t* trace_off;    /* [ntraces+1] start of each trace in `traces`            */
    const float*   half_offset;  /* [ntraces] h = |receiver - source| / 2 (m)              */
    const float*   midpoint;     /* [ntraces] CDP midpoint (m); may be NULL for CMP calls  */
    const int64_t* gather_off;   /* [ngathers+1] traces of gather g                        */
    const int64_t* out_off;      /* [ngathers+1] output rows of gather g                   */
    const float*   dt;           /* [ngathers] sampling interval of gather g (s)           */
    int64_t ngathers;            /* host value                                             */
    int64_t ntraces;             /* host value                                             */
    int32_t max_rows;            /* host: >= out_off[g+1]-out_off[g] for every g           */
    int32_t max_trace_samples;   /* host: >= trace_off[i+1]-trace_off[i] for every i       */
} seis_gathers;

/* CRS apertures (Section 2.2, Section 3.5): for each central CDP c the traces of every
 * CDP whose midpoint lies within the aperture radius, and the central's own output
 * grid.  Built by seis_crs_aperture() or by the caller. */
typedef struct seis_aperture {
    const int64_t* nbr_off;      /* [n_central+1] entries of central c in nbr_trace       */
    const int32_t* nbr_trace;    /* [nbr_off[n_central]] trace indices                     */
    const float*   m_c;          /* [n_central] central midpoint (m); dm = midpoint - m_c  */
    const int64_t* out_off;      /* [n_central+1] output rows of central c                 */
    const float*   dt;           /* [n_central] sampling interval of central c (s)         */
    int64_t n_central;           /* host value                                             */
    int32_t max_rows;            /* host: >= out_off[c+1]-out_off[c] for every c           */
    int32_t pad_;
} seis_aperture;

/* Message describing the last failure on the calling thread ("" if none). */
const char* seis_last_error(void);

/* SYNCHRONOUS.  Waits for `stream`, then reports (and clears) what kernels of this library
 * recorded in the device status word since the last call: SEIS_ETIMEOUT (a bounded device
 * wait gave up), SEIS_EUNSUPPORTED (a staged window overflowed), SEIS_EINVAL (a batch item
 * was skipped), else SEIS_OK. */
int seis_device_status(void* stream);

/* Self-test of the bounded device waits (no counterpart in the paper).  Launches one CTA
 * that waits on a shared-memory mbarrier nothing completes, through the same bounded wait
 * as the search kernels but with a limit of limit_us microseconds (1 .. 1e6); the wait
 * gives up, records SEIS_ETIMEOUT in the device status word and the kernel returns, so the
 * next seis_device_status() reports it and the context stays usable. */
int seis_selftest_wait_timeout(int32_t limit_us, void* stream);

/* Self-test of the fast arithmetic of the traveltime (no counterpart in the paper, which
 * takes the square root of Eq. 2's traveltime exactly): the search, t0-window and
 * evaluation kernels form u = sqrt(radicand) and 1/(u + p) with the hardware's approximate
 * square root and reciprocal (PTX sqrt.approx.ftz.f32, rcp.approx.ftz.f32).  This runs both
 * on every float in [1, 4) (all mantissas under both exponent parities; the relative error
 * repeats with the exponent) and writes, to max_rel_err[0] and [1] (device, 2 floats,
 * caller-owned), the largest relative error of each against an FP64 reference.
 * Asynchronous, one launch.  Errors: SEIS_EINVAL, SEIS_ECUDA. */
int seis_selftest_fast_math(float* max_rel_err, void* stream);

/* Search kernel variants.  The semblance search kernels come in several tile shapes and
 * arithmetic forms (consumer warps per CTA, candidates per thread, scalar / packed f32x2 /
 * hybrid FP32 accumulation); every variant computes bit-identical results.  A launch uses
 * the variant the autotuner recorded for its shape bucket (kind, w, and log2 buckets of
 * the candidate count, rows per owner and traces per gather), else the process-wide
 * default set here (initially 4).  Changing it while other host threads launch searches is
 * allowed; those launches use either value. */
int seis_search_variant_count(void);
const char* seis_search_variant_name(int variant);      /* "" if out of range */
int seis_set_search_variant(int variant);                /* SEIS_EINVAL if out of range */
int seis_get_search_variant(void);

/* Autotuner (no counterpart in the paper; it picks the tile shape the paper fixes by hand
 * for the Sunway LDM, Section 3.3.2 "tile_size").  SYNCHRONOUS: runs every variant once
 * untimed and `reps` times between CUDA events on `stream`, records the fastest for the
 * problem's shape bucket and returns it in *chosen (host, may be NULL); ms_out (host,
 * seis_search_variant_count() floats, may be NULL) receives each variant's mean time.
 * best_idx / best_S / stack_out are scratch outputs of the problem's size (overwritten).
 * Arguments as cmp_semblance / crs_semblance; errors likewise. */
int seis_autotune_cmp(const seis_gathers* d, const float* C, int32_t nc, int32_t w,
                      int32_t* best_idx, float* best_S, float* stack_out, int32_t reps,
                      int32_t* chosen, float* ms_out, void* stream);
int seis_autotune_crs(const seis_gathers* d, const seis_aperture* ap,
                      const float* A, int32_t nA, const float* B, int32_t nB,
                      const float* C, int32_t nC, int32_t w,
                      int32_t* best_idx, float* best_S, float* stack_out, int32_t reps,
                      int32_t* chosen, float* ms_out, void* stream);
/* The recorded choices as a JSON file (host path); load merges into the current table. */
int seis_autotune_save(const char* path);
int seis_autotune_load(const char* path);
int seis_autotune_clear(void);

/* Candidate grid of the CMP search -- Section 3.2 (the NMO velocity array is generated
 * from its lower and upper bounds): nc velocities linearly spaced over [vmin, vmax] m/s,
 * both bounds included (nc = 1 gives vmin alone), written as C = 4/v^2 (s^2/m^2), the
 * parameter of the hyperbola t^2 = t0^2 + C h^2 in half-offset h (Section 2.1).  Each value
 * is formed in FP64 and rounded once to FP32.
 *   C_out [nc] device, caller-owned.  Asynchronous, one launch.
 * Errors: SEIS_EINVAL (C_out NULL, nc < 1, a bound not finite or not positive), SEIS_ECUDA. */
int seis_velocity_grid(double vmin, double vmax, int32_t nc, float* C_out, void* stream);

/* A linear parameter axis: n values lo + (hi - lo) i / (n - 1), i = 0 .. n-1, both ends
 * included (n = 1 gives lo), formed in FP64 and rounded once to FP32 -- the A, B and C axes
 * of the CRS search (Section 2.2; the flattened grid of crs_semblance).
 *   out [n] device, caller-owned.  Asynchronous, one launch.
 * Errors: SEIS_EINVAL (out NULL, n < 1, a bound not finite), SEIS_ECUDA. */
int seis_linear_grid(double lo, double hi, int32_t n, float* out, void* stream);

/* CMP semblance search -- Section 2.1, Eq. 1, Algorithm 1, Section 3.2.
 * For every output row (gather g, t0 = n*dt[g]) and every candidate C[c] (C = 4/v^2,
 * s^2/m^2) each trace of gather g is intersected at t = sqrt(t0^2 + C h^2), its
 * amplitude linearly interpolated along the window, and the windowed semblance formed.
 *   C          [nc] candidates (any order; typically 4/v^2 of a linear velocity grid)
 *   S_cube     [rows][nc] semblance of every (row, candidate), or NULL
 *   best_idx   [rows] argmax candidate index
 *   best_C     [rows] C[best_idx], or NULL
 *   best_S     [rows] semblance at the argmax
 *   stack_out  [rows] stack along the picked curve (Algorithm 1's linear accumulator)
 * rows = out_off[ngathers].  Errors: SEIS_EINVAL (null pointer, nc < 1, w even or out of
 * range, max_trace_samples above SEIS_MAX_TRACE_SAMPLES), SEIS_ECUDA. */
int cmp_semblance(const seis_gathers* d, const float* C, int32_t nc, int32_t w,
                  float* S_cube, int32_t* best_idx, float* best_C, float* best_S,
                  float* stack_out, void* stream);

/* CMP semblance with the window over neighbouring output times (not the paper's method:
 * Algorithm 1 windows along each trace around its own intersection).  For output time
 * t0 = n dt and candidate C, the window runs over t0' = t0 + j dt (j = -hw..hw, rows of
 * the same gather only), each with its own traveltime t = sqrt(t0'^2 + C h^2) (Section
 * 2.1), and every trace gives one linearly interpolated sample v there; a trace takes part
 * at t0' when both interpolation samples lie inside it.  With s, e, M the sum of v, of v^2
 * and the count of traces taking part at t0':
 *   S = sum_j s(t0')^2 / sum_j M(t0') e(t0')   (0 if the denominator is 0),
 * stack_out = s(t0) / M(t0) at the pick.  Arguments, layouts and errors as cmp_semblance
 * (one launch; no workspace). */
int cmp_semblance_t0win(const seis_gathers* d, const float* C, int32_t nc, int32_t w,
                        float* S_cube, int32_t* best_idx, float* best_C, float* best_S,
                        float* stack_out, void* stream);

/* CRS semblance with the window over neighbouring output times: cmp_semblance_t0win's
 * definition with the CRS traveltime t = sqrt((t0' + A dm)^2 + B dm^2 + C h^2) of Section
 * 2.2 over the aperture's traces (a trace also needs t0' + A dm >= 0 and a real t).
 * Arguments, layouts and errors as crs_semblance (one launch; no workspace). */
int crs_semblance_t0win(const seis_gathers* d, const seis_aperture* ap, const float* A,
                        int32_t nA, const float* B, int32_t nB, const float* C, int32_t nC,
                        int32_t w, float* S_cube, int32_t* best_idx, float* best_ABC,
                        float* best_S, float* stack_out, void* stream);

/* CRS aperture build -- Section 2.2 (the central CDP uses the traces of the CDPs within
 * radius r) and Section 3.5 (each CDP draws a circle around its midpoint).  For each
 * central gather central[c] (device int32 [n_central]) lists, in increasing order, every
 * trace i with |midpoint[i] - midpoint[first trace of central[c]]| <= apm (inclusive),
 * and fills m_c, out_off (rows of the central gathers, concatenated) and dt.
 * SYNCHRONOUS.  Call once with nbr_trace == NULL to fill nbr_off and learn
 * *total_entries (host); then call again with nbr_trace of at least that capacity.
 *   nbr_off [n_central+1], m_c [n_central], out_off [n_central+1], dt_c [n_central] device
 *   total_entries, total_rows, max_rows: host outputs (may be NULL)
 * Errors: SEIS_EINVAL (null pointers, apm < 0, a central index out of range or empty,
 * capacity too small), SEIS_ECUDA. */
int seis_crs_aperture(const seis_gathers* d, const int32_t* central, int64_t n_central,
                      float apm, int64_t* nbr_off, int32_t* nbr_trace, int64_t capacity,
                      float* m_c, int64_t* out_off, float* dt_c,
                      int64_t* total_entries, int64_t* total_rows, int32_t* max_rows,
                      void* stream);

/* As seis_crs_aperture, keeping only the traces with |half_offset| <= hmax (hmax >= 0; 0
 * keeps the zero-offset traces), e.g. for the zero-offset stage of crs_pragmatic.  Errors as
 * seis_crs_aperture, and SEIS_EINVAL for hmax < 0 or NaN. */
int seis_crs_aperture_offset(const seis_gathers* d, const int32_t* central, int64_t n_central,
                             float apm, float hmax, int64_t* nbr_off, int32_t* nbr_trace,
                             int64_t capacity, float* m_c, int64_t* out_off, float* dt_c,
                             int64_t* total_entries, int64_t* total_rows, int32_t* max_rows,
                             void* stream);

/* The searches for problems too small to fill the GPU (no counterpart in the paper, whose
 * CGs take one CDP each, Section 3.5).  A search launches one CTA per (gather or central
 * CDP, tile of 32 output rows), so a few owners leave most SMs idle, and a grid just past a
 * whole number of waves leaves a last wave nearly empty.  These entry points split each
 * tile's candidates over the fewest CTAs that keep at least 90 % of the launch's waves
 * occupied (two CTAs per SM), each CTA writing the argmax of its own candidates to the
 * workspace, and merge the parts per row (the earlier part on ties).  A split launch uses
 * the default kernel variant (4) whatever the autotuner recorded.  Every output is
 * bit-identical to cmp_semblance / crs_semblance; with enough tiles they run exactly those.
 *   workspace: device scratch of seis_search_workspace_size(n_owner, max_rows, rows, ncand)
 *   bytes (0 when no split is needed; then workspace may be NULL), 16-byte aligned,
 *   caller-owned; n_owner = ngathers (CMP) or ap->n_central (CRS), max_rows and ncand as in
 *   the call, rows (host) = the number of output rows (out_off[n_owner]).  The split depends
 *   on the current device's SM count.
 * Other arguments, outputs and errors as cmp_semblance / crs_semblance, and SEIS_EINVAL
 * when the workspace is too small. */
size_t seis_search_workspace_size(int64_t n_owner, int32_t max_rows, int64_t rows,
                                  int64_t ncand);
int cmp_semblance_ws(const seis_gathers* d, const float* C, int32_t nc, int32_t w,
                     float* S_cube, int32_t* best_idx, float* best_C, float* best_S,
                     float* stack_out, void* workspace, size_t ws_bytes, int64_t rows,
                     void* stream);
int crs_semblance_ws(const seis_gathers* d, const seis_aperture* ap, const float* A,
                     int32_t nA, const float* B, int32_t nB, const float* C, int32_t nC,
                     int32_t w, float* S_cube, int32_t* best_idx, float* best_ABC,
                     float* best_S, float* stack_out, void* workspace, size_t ws_bytes,
                     int64_t rows, void* stream);

/* CRS semblance search -- Section 2.2, Section 3.5 (aperture), Eq. 1, Algorithm 1.
 * Candidates are the flattened grid cand = (ia*nB + ib)*nC + ic of A[nA] (s/m),
 * B[nB] (s^2/m^2), C[nC] (s^2/m^2); trace i of the aperture of central c is intersected
 * at t = sqrt((t0 + A dm)^2 + B dm^2 + C h^2), dm = midpoint[i] - m_c[c].
 *   S_cube     [rows][nA*nB*nC] or NULL
 *   best_idx   [rows] flattened argmax
 *   best_ABC   [rows][3] (A, B, C) at the argmax, or NULL
 *   best_S, stack_out [rows]
 * rows = ap->out_off[n_central].  d->midpoint must be set.  Errors as cmp_semblance. */
int crs_semblance(const seis_gathers* d, const seis_aperture* ap,
                  const float* A, int32_t nA, const float* B, int32_t nB,
                  const float* C, int32_t nC, int32_t w,
                  float* S_cube, int32_t* best_idx, float* best_ABC, float* best_S,
                  float* stack_out, void* stream);

/* Stack along given operators -- Algorithm 1's linear accumulator (stack = sum of the
 * interpolated window samples / (N w)), Section 2.1 (NMO correction and stacking).
 * ap == NULL: CMP mode, params [rows] = C per output row of the gathers in d.
 * ap != NULL: CRS mode, params [rows][3] = (A, B, C) per output row of the apertures.
 *   stack_out [rows]; S_out [rows] semblance at the operator (or NULL); N_out [rows] number
 *   of traces taking part (or NULL).  Errors: SEIS_EINVAL, SEIS_ECUDA. */
int stack(const seis_gathers* d, const seis_aperture* ap, const float* params, int32_t w,
          float* stack_out, float* S_out, int32_t* N_out, void* stream);

/* Adjoint of the CRS semblance (no counterpart in the paper: the derivative of Eq. 1
 * through the CRS traveltime of Section 2.2 and the linear interpolation of Algorithm 1,
 * with k and the participation mask held fixed).  For ABC [rows][3] gives S_out [rows],
 * grad_out [rows][3] = dS/d(A,B,C) and, if non-NULL, stack_out [rows]. */
int crs_semblance_grad(const seis_gathers* d, const seis_aperture* ap, const float* ABC,
                       int32_t w, float* S_out, float* grad_out, float* stack_out, void* stream);

/* Gradient-ascent refinement of the CRS operators (no counterpart in the paper; it replaces
 * the dense 3-D grid search of Section 2.2 by a local search from a coarse pick).  Per row,
 * in normalised coordinates z = (theta - lo3) / (hi3 - lo3), with g = dS/dz: starting from
 * ABC_inout, `steps` projected quasi-Newton trials z' = clamp(z + a d, 0, 1), d = H g, where H
 * (the inverse-curvature estimate, BFGS-updated after each accepted trial) starts as
 * (step0/|g|) I and |d| is capped at 0.25; a trial is accepted when its S is not lower, and a
 * rejected trial halves a (a = 1 after each acceptance).  On return ABC_inout holds the accepted
 * operators and S_out, grad_out [rows][3], stack_out their semblance, gradient and stack.
 * lo3, hi3: HOST arrays of 3 floats.  rows = ap->out_off[n_central] (host).  workspace:
 * device scratch of seis_refine_workspace_size(rows) bytes, 256-byte aligned, owned by the
 * caller.  Asynchronous (1 + 2*steps launches on stream).  Errors: SEIS_EINVAL, SEIS_ECUDA. */
size_t seis_refine_workspace_size(int64_t rows);
int crs_refine(const seis_gathers* d, const seis_aperture* ap, float* ABC_inout,
               const float* lo3, const float* hi3, int32_t steps, float step0, int32_t w,
               float* S_out, float* grad_out, float* stack_out,
               void* workspace, size_t ws_bytes, int64_t rows, void* stream);

/* Starting points for a multi-start refinement (no counterpart in the paper): from a coarse
 * CRS semblance cube S_cube [rows][nA*nB*nC] (device, as crs_semblance writes it, candidate
 * cand = (ia*nB + ib)*nC + ic), the nstart best candidates of every row in the order
 * S descending, candidate index ascending on ties, decoded to ABC_starts [nstart][rows][3]
 * (device, caller-owned; start j of row r at (j*rows + r)*3).  A, B, C: device axes.
 * 1 <= nstart <= nA*nB*nC.  Asynchronous, one launch.  Errors: SEIS_EINVAL, SEIS_ECUDA. */
int crs_top_starts(const float* S_cube, int64_t rows, const float* A, int32_t nA,
                   const float* B, int32_t nB, const float* C, int32_t nC, int32_t nstart,
                   float* ABC_starts, void* stream);

/* Starting points at the local maxima of the coarse cube (no counterpart in the paper): as
 * crs_top_starts, but a row's starts are first its local maxima -- candidates whose
 * (S, -index) exceeds that of every neighbour in the grid (ia, ib, ic each within +-1, up to
 * 26 neighbours) -- in the order S descending, index ascending, and only then, if the row
 * has fewer than nstart local maxima, its best other candidates in that order.  Starts at
 * distinct local maxima climb distinct hills of S, where the nstart best candidates often
 * crowd around one.  nA*nB*nC <= SEIS_LOCAL_MAX_CANDIDATES (SEIS_EUNSUPPORTED beyond).
 * Arguments, layout and errors otherwise as crs_top_starts (one launch). */
#define SEIS_LOCAL_MAX_CANDIDATES 32768
int crs_local_max_starts(const float* S_cube, int64_t rows, const float* A, int32_t nA,
                         const float* B, int32_t nB, const float* C, int32_t nC,
                         int32_t nstart, float* ABC_starts, void* stream);

/* Multi-start refinement (no counterpart in the paper): crs_refine from each of the nstart
 * starting operators ABC_starts [nstart][rows][3] (device, read only), keeping per row the
 * result with the highest S (the earlier start on ties) in ABC_out [rows][3], S_out,
 * grad_out [rows][3] and stack_out [rows].  Other arguments as crs_refine; workspace:
 * seis_refine_multi_workspace_size(rows) bytes, 256-byte aligned, caller-owned.
 * Asynchronous (nstart * (3 + 2*steps) operations on stream).  Errors: SEIS_EINVAL,
 * SEIS_ECUDA. */
size_t seis_refine_multi_workspace_size(int64_t rows);
int crs_refine_multi(const seis_gathers* d, const seis_aperture* ap, const float* ABC_starts,
                     int32_t nstart, const float* lo3, const float* hi3, int32_t steps,
                     float step0, int32_t w, float* ABC_out, float* S_out, float* grad_out,
                     float* stack_out, void* workspace, size_t ws_bytes, int64_t rows,
                     void* stream);

/* CRS operator by two small searches instead of the dense grid (not in the paper, which
 * searches the dense A x B x C grid of Section 2.2): C from the central CMP's own traces
 * (ap_cmp: apm = 0, so dm = 0 and the traveltime is the CMP one of Section 2.1; A = B = 0),
 * then A and B from the zero-offset traces of the aperture (ap_zo: seis_crs_aperture_offset
 * with a small hmax; the C term is taken at the single value c_zo and vanishes where h = 0),
 * then S and the stack of the combined operator (A, B from the second search, C from the
 * first) over the full aperture ap_full, as stack() computes them.  The three apertures
 * describe the same central CDPs (same n_central and rows).  Outputs best_ABC [rows][3],
 * best_S, stack_out [rows] (device).  workspace: seis_pragmatic_workspace_size(rows) bytes,
 * 256-byte aligned, caller-owned.  Asynchronous (two searches, the stack and two small
 * kernels on stream).  Errors: SEIS_EINVAL, SEIS_ECUDA. */
size_t seis_pragmatic_workspace_size(int64_t rows);
int crs_pragmatic(const seis_gathers* d, const seis_aperture* ap_full,
                  const seis_aperture* ap_cmp, const seis_aperture* ap_zo, const float* A,
                  int32_t nA, const float* B, int32_t nB, const float* C, int32_t nC, float c_zo,
                  int32_t w, float* best_ABC, float* best_S, float* stack_out, void* workspace,
                  size_t ws_bytes, int64_t rows, void* stream);

/* Batched search (no counterpart in the paper: its CGs take one CDP per task, Section 3.5;
 * here thousands of uneven CMP gathers and CRS supergathers run in ONE persistent launch
 * that can be captured in a CUDA graph).  Item i owns the traces
 * [trace_begin, trace_end) of d (a CRS item's traces carry their own midpoints, so the
 * item is its own aperture), the output rows [out_begin, out_begin + rows) at t0 = n*dt,
 * and the candidate axes A = poolA[a_off .. a_off+nA), B = poolB[b_off ..), C = poolC[c_off
 * ..) searched as cand = (ia*nB + ib)*nC + ic (CMP items: nA = nB = 1, A and B ignored).
 * Results as crs_semblance (best_ABC holds (0, 0, C) for CMP items).  Items with an
 * out-of-range field are skipped and flagged in the device status word. */
typedef struct seis_batch_item {
    int64_t trace_begin, trace_end;
    int64_t out_begin;
    int32_t rows;
    int32_t kind;            /* 0 = CMP gather, 1 = CRS supergather */
    float   dt;              /* s */
    float   m_c;             /* CRS: central midpoint (m) */
    int32_t a_off, nA;
    int32_t b_off, nB;
    int32_t c_off, nC;
} seis_batch_item;

/* Device scratch of seis_batch_workspace_size(nitems) bytes (256-byte aligned, caller-owned)
 * holds the work counter and the task table; every call rebuilds it.
 *   items: device [nitems]; pool sizes are host values used for the range checks;
 *   out_rows (host) = length of the output arrays (best_ABC: 3 * out_rows floats).
 *   mode 0: one persistent launch (grid = 2 CTAs per SM, tasks claimed from the counter);
 *   mode 1: one launch per item (the comparison; SYNCHRONOUS: reads the item table back).
 * d: traces, trace_off, half_offset, midpoint (needed when an item is CRS); gather fields
 * are not used.  Errors: SEIS_EINVAL, SEIS_ECUDA. */
size_t seis_batch_workspace_size(int64_t nitems);
int seis_batch_semblance(const seis_gathers* d, const seis_batch_item* items, int64_t nitems,
                         const float* poolA, int32_t sizeA, const float* poolB, int32_t sizeB,
                         const float* poolC, int32_t sizeC, int32_t w, int32_t mode,
                         int32_t* best_idx, float* best_ABC, float* best_S, float* stack_out,
                         int64_t out_rows, void* workspace, size_t ws_bytes, void* stream);

/* Autotuner of the batched search (no counterpart in the paper): runs the persistent
 * launch of seis_batch_semblance once untimed and `reps` times between CUDA events with each
 * variant the batch kernel is built for (0, 1, 3, 4, 9, 10), records the fastest for the
 * window length w (later seis_batch_semblance calls with that w use it) and returns it in
 * *chosen (host, may be NULL).  ms_out (host, seis_search_variant_count() floats, may be
 * NULL) receives each tried variant's mean time and -1 for the others.  SYNCHRONOUS.
 * Arguments, outputs and errors as seis_batch_semblance (mode 0). */
int seis_autotune_batch(const seis_gathers* d, const seis_batch_item* items, int64_t nitems,
                        const float* poolA, int32_t sizeA, const float* poolB, int32_t sizeB,
                        const float* poolC, int32_t sizeC, int32_t w, int32_t* best_idx,
                        float* best_ABC, float* best_S, float* stack_out, int64_t out_rows,
                        void* workspace, size_t ws_bytes, int32_t reps, int32_t* chosen,
                        float* ms_out, void* stream);

/* Allocation-free batched search (the paper has no counterpart: it concerns how this
 * library is called, not the method).  For callers that cannot allocate device memory
 * where they call the library -- a service running under a fixed device-memory budget, a
 * plug-in whose host application owns all allocations, a latency-bound loop that cannot
 * afford cudaMalloc's possible device synchronisation -- this runs seis_batch_semblance in
 * its persistent mode (mode 0) with the scratch (work counter and task table) kept in a
 * device array inside the library instead of a caller workspace.  Limits and behaviour:
 *   - at most SEIS_NOALLOC_MAX_ITEMS items per call (SEIS_EINVAL beyond); the array,
 *     seis_batch_workspace_size(SEIS_NOALLOC_MAX_ITEMS) = 524,800 bytes (about 512 KiB),
 *     is held on every GPU that loads the library until the process exits;
 *   - the first call on a device looks the array's device address up (a runtime query,
 *     not an allocation) and keeps it, so make that first call before any stream capture,
 *     and do not call this entry point on a device after cudaDeviceReset() in the same
 *     process (the kept address belongs to the context the reset destroyed);
 *   - every call shares the array (each rebuilds the task table and zeroes the counter):
 *     calls whose work overlaps on the GPU race on it, so serialise them;
 *   - nothing is allocated: no cudaMalloc, no cudaFree, no allocating library routine.
 * Arguments and results as seis_batch_semblance. */
#define SEIS_NOALLOC_MAX_ITEMS 65536
int seis_batch_semblance_noalloc(const seis_gathers* d, const seis_batch_item* items,
                                 int64_t nitems, const float* poolA, int32_t sizeA,
                                 const float* poolB, int32_t sizeB, const float* poolC,
                                 int32_t sizeC, int32_t w, int32_t* best_idx, float* best_ABC,
                                 float* best_S, float* stack_out, int64_t out_rows, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SEIS_H */
