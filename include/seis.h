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
 *   - Kernels never read or write outside the arrays described here, whatever the
 *     contents of the offset arrays; inconsistent offsets give unspecified results.
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

/* SYNCHRONOUS.  Waits for `stream`, then returns SEIS_OK, or SEIS_ETIMEOUT if a kernel of
 * this library recorded a timed-out device wait since the last call (and clears it). */
int seis_device_status(void* stream);

/* Search kernel variants.  The semblance search kernels come in several tile shapes and
 * arithmetic forms (consumer warps per CTA, candidates per thread, packed f32x2 or scalar
 * FP32 accumulation); every variant computes bit-identical results.  The variant used by
 * cmp_semblance / crs_semblance is a process-wide setting (default 0), normally chosen by
 * the autotuner (seis_autotune_cmp); changing it while other host threads launch searches
 * is allowed but those launches may use either value. */
int seis_search_variant_count(void);
const char* seis_search_variant_name(int variant);      /* "" if out of range */
int seis_set_search_variant(int variant);                /* SEIS_EINVAL if out of range */
int seis_get_search_variant(void);

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

#ifdef __cplusplus
}
#endif
#endif /* SEIS_H */
