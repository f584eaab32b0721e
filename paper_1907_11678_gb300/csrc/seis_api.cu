// seis_api.cu -- the C ABI of libseis (declared in include/seis.h): argument checks,
// error reporting, the device status word, and the CRS aperture build.
#include <cmath>
#include <cuda_runtime.h>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>
#include "seis.h"
#include "seis_dev.cuh"
#include "seis_internal.h"

namespace seis {

// ------------------------------------------------------------------ error reporting --
static thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(SEIS_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// --------------------------------------------------------------- device status word --
__device__ unsigned g_status;

unsigned* device_status_word() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    return static_cast<unsigned*>(p);
}

static bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

static int check_gathers(const seis_gathers* d, bool need_midpoint) {
    if (!d) return fail(SEIS_EINVAL, "gathers descriptor is NULL");
    if (!d->traces || !d->trace_off || !d->half_offset || !d->gather_off || !d->out_off || !d->dt)
        return fail(SEIS_EINVAL, "a required gathers array is NULL");
    if (need_midpoint && !d->midpoint) return fail(SEIS_EINVAL, "midpoint array is NULL");
    if (!aligned4(d->traces)) return fail(SEIS_EINVAL, "traces must be 4-byte aligned");
    if (d->ngathers < 1 || d->ntraces < 0) return fail(SEIS_EINVAL, "ngathers must be >= 1");
    if (d->max_rows < 1) return fail(SEIS_EINVAL, "max_rows must be >= 1");
    if (d->max_trace_samples < 0 || d->max_trace_samples > SEIS_MAX_TRACE_SAMPLES)
        return fail(SEIS_EINVAL, "max_trace_samples %d outside [0, %d]", d->max_trace_samples,
                    SEIS_MAX_TRACE_SAMPLES);
    return SEIS_OK;
}

static int check_w(int32_t w) {
    if (w < 1 || (w % 2) == 0 || w > SEIS_MAX_W)
        return fail(SEIS_EINVAL, "window w = %d must be odd and in [1, %d]", w, SEIS_MAX_W);
    return SEIS_OK;
}

// Variant used where the autotuner has no entry: 4 (15 warps x 2 candidates, packed f32x2),
// the fastest on every CMP and CRS workload measured.
static std::atomic<int> g_variant{4};

int default_variant() { return g_variant.load(); }

int build_cmp_params(const seis_gathers* d, const float* C, int32_t nc, int32_t w, float* S_cube,
                     int32_t* best_idx, float* best_C, float* best_S, float* stack_out,
                     SearchParams* out, TuneKey* key) {
    int rc = check_gathers(d, false);
    if (rc) return rc;
    if ((rc = check_w(w))) return rc;
    if (!C || nc < 1) return fail(SEIS_EINVAL, "C must be non-NULL with nc >= 1");
    if (!best_idx || !best_S || !stack_out) return fail(SEIS_EINVAL, "an output array is NULL");
    SearchParams p{};
    p.traces = d->traces;
    p.trace_off = d->trace_off;
    p.h = d->half_offset;
    p.m = nullptr;
    p.list_off = d->gather_off;
    p.list = nullptr;
    p.m_c = nullptr;
    p.out_off = d->out_off;
    p.dt = d->dt;
    p.nowner = d->ngathers;
    p.tiles_per_owner = (d->max_rows + 31) / 32;
    p.A = nullptr;
    p.B = nullptr;
    p.C = C;
    p.nA = 1;
    p.nB = 1;
    p.nC = nc;
    p.ncand = nc;
    p.S_cube = S_cube;
    p.best_idx = best_idx;
    p.best_param = best_C;
    p.best_S = best_S;
    p.stack = stack_out;
    p.status = device_status_word();
    p.nsplit = 1;
    p.partial = nullptr;
    *key = make_tune_key(false, w, nc, d->max_rows, d->ntraces / d->ngathers);
    p.variant = lookup_variant(*key, default_variant());
    *out = p;
    return SEIS_OK;
}

int build_crs_params(const seis_gathers* d, const seis_aperture* ap, const float* A, int32_t nA,
                     const float* B, int32_t nB, const float* C, int32_t nC, int32_t w,
                     float* S_cube, int32_t* best_idx, float* best_ABC, float* best_S,
                     float* stack_out, SearchParams* out, TuneKey* key) {
    int rc = check_gathers(d, true);
    if (rc) return rc;
    if ((rc = check_w(w))) return rc;
    if (!ap || !ap->nbr_off || !ap->nbr_trace || !ap->m_c || !ap->out_off || !ap->dt)
        return fail(SEIS_EINVAL, "aperture descriptor or one of its arrays is NULL");
    if (ap->n_central < 1 || ap->max_rows < 1)
        return fail(SEIS_EINVAL, "aperture needs n_central >= 1 and max_rows >= 1");
    if (!A || !B || !C || nA < 1 || nB < 1 || nC < 1)
        return fail(SEIS_EINVAL, "A, B, C must be non-NULL with nA, nB, nC >= 1");
    const int64_t ncand = (int64_t)nA * nB * nC;
    if (ncand > (int64_t)1 << 30) return fail(SEIS_EINVAL, "too many candidates");
    if (!best_idx || !best_S || !stack_out) return fail(SEIS_EINVAL, "an output array is NULL");
    SearchParams p{};
    p.traces = d->traces;
    p.trace_off = d->trace_off;
    p.h = d->half_offset;
    p.m = d->midpoint;
    p.list_off = ap->nbr_off;
    p.list = ap->nbr_trace;
    p.m_c = ap->m_c;
    p.out_off = ap->out_off;
    p.dt = ap->dt;
    p.nowner = ap->n_central;
    p.tiles_per_owner = (ap->max_rows + 31) / 32;
    p.A = A;
    p.B = B;
    p.C = C;
    p.nA = nA;
    p.nB = nB;
    p.nC = nC;
    p.ncand = (int)ncand;
    p.S_cube = S_cube;
    p.best_idx = best_idx;
    p.best_param = best_ABC;
    p.best_S = best_S;
    p.stack = stack_out;
    p.status = device_status_word();
    p.nsplit = 1;
    p.partial = nullptr;
    *key = make_tune_key(true, w, (int)ncand, ap->max_rows, 0);
    p.variant = lookup_variant(*key, default_variant());
    *out = p;
    return SEIS_OK;
}

}  // namespace seis

using namespace seis;

extern "C" const char* seis_last_error(void) { return g_err; }

extern "C" int seis_search_variant_count(void) { return search_variant_count(); }

extern "C" const char* seis_search_variant_name(int variant) { return search_variant_name(variant); }

extern "C" int seis_set_search_variant(int variant) {
    if (variant < 0 || variant >= search_variant_count())
        return fail(SEIS_EINVAL, "variant %d outside [0, %d)", variant, search_variant_count());
    g_variant.store(variant);
    return SEIS_OK;
}

extern "C" int seis_get_search_variant(void) { return g_variant.load(); }

extern "C" int seis_device_status(void* stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "seis_device_status");
    unsigned v = 0, zero = 0;
    e = cudaMemcpyFromSymbol(&v, g_status, sizeof(v));
    if (e != cudaSuccess) return cuda_fail(e, "seis_device_status");
    e = cudaMemcpyToSymbol(g_status, &zero, sizeof(zero));
    if (e != cudaSuccess) return cuda_fail(e, "seis_device_status");
    if (v & kStatusTimeout) return fail(SEIS_ETIMEOUT, "a device wait timed out");
    if (v & kStatusOverflow) return fail(SEIS_EUNSUPPORTED, "a staged trace window overflowed");
    if (v & kStatusBadItem) return fail(SEIS_EINVAL, "a batch item with an out-of-range field was skipped");
    return SEIS_OK;
}

extern "C" int cmp_semblance(const seis_gathers* d, const float* C, int32_t nc, int32_t w,
                             float* S_cube, int32_t* best_idx, float* best_C, float* best_S,
                             float* stack_out, void* stream) {
    SearchParams p;
    TuneKey key;
    int rc = build_cmp_params(d, C, nc, w, S_cube, best_idx, best_C, best_S, stack_out, &p, &key);
    if (rc) return rc;
    cudaError_t e = launch_search(p, false, w, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cmp_semblance launch");
    return SEIS_OK;
}

extern "C" int crs_semblance(const seis_gathers* d, const seis_aperture* ap, const float* A,
                             int32_t nA, const float* B, int32_t nB, const float* C, int32_t nC,
                             int32_t w, float* S_cube, int32_t* best_idx, float* best_ABC,
                             float* best_S, float* stack_out, void* stream) {
    SearchParams p;
    TuneKey key;
    int rc = build_crs_params(d, ap, A, nA, B, nB, C, nC, w, S_cube, best_idx, best_ABC, best_S,
                              stack_out, &p, &key);
    if (rc) return rc;
    cudaError_t e = launch_search(p, true, w, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "crs_semblance launch");
    return SEIS_OK;
}

// ------------------------------------------------------------------ aperture build ----
namespace seis {

// One CTA per central CDP: validate it (count -1 if the index is out of range or the
// gather is empty), record its midpoint, rows and dt, and count the traces inside its
// aperture (|m_i - m_c| <= apm in FP64, inclusive, and |h_i| <= hmax).
__global__ void aperture_count_kernel(const float* m, const float* h, const int64_t* gather_off,
                                      const int64_t* out_off, const float* dt, int64_t ngathers,
                                      int64_t ntraces, const int32_t* central, float apm,
                                      float hmax, int64_t* counts, float* m_c, int64_t* rows,
                                      float* dt_c) {
    const int64_t c = blockIdx.x;
    const int32_t g = central[c];
    __shared__ unsigned long long part[256];
    if (g < 0 || g >= ngathers || gather_off[g + 1] <= gather_off[g]) {
        if (threadIdx.x == 0) { counts[c] = -1; rows[c] = 0; m_c[c] = 0.f; dt_c[c] = 0.f; }
        return;
    }
    const float mg = m[gather_off[g]];
    unsigned long long cnt = 0;
    for (int64_t i = threadIdx.x; i < ntraces; i += blockDim.x)
        cnt += (fabs((double)m[i] - (double)mg) <= (double)apm && fabsf(h[i]) <= hmax) ? 1ull
                                                                                       : 0ull;
    part[threadIdx.x] = cnt;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        counts[c] = (int64_t)part[0];
        m_c[c] = mg;
        rows[c] = out_off[g + 1] - out_off[g];
        dt_c[c] = dt[g];
    }
}

// One CTA per central CDP: ordered compaction of the aperture's trace indices.
__global__ void aperture_fill_kernel(const float* m, const float* h, int64_t ntraces,
                                     const int64_t* nbr_off, const float* m_c, float apm,
                                     float hmax, int32_t* nbr_trace) {
    const int64_t c = blockIdx.x;
    const double mg = (double)m_c[c];
    __shared__ int wsum[8];
    int64_t base = nbr_off[c];
    const int64_t end = nbr_off[c + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i0 = 0; i0 < ntraces; i0 += 256) {
        const int64_t i = i0 + threadIdx.x;
        const bool in = i < ntraces && fabs((double)m[i] - mg) <= (double)apm &&
                        fabsf(h[i]) <= hmax;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w2 = 0; w2 < 8; ++w2) {
            if (w2 < warp) before += wsum[w2];
            total += wsum[w2];
        }
        const int pos = before + __popc(bal & ((1u << lane) - 1u));
        if (in && base + pos < end) nbr_trace[base + pos] = (int32_t)i;
        base += total;
        __syncthreads();
    }
}

}  // namespace seis

static int crs_aperture_impl(const seis_gathers* d, const int32_t* central, int64_t n_central,
                             float apm, float hmax, int64_t* nbr_off, int32_t* nbr_trace,
                             int64_t capacity, float* m_c, int64_t* out_off, float* dt_c,
                             int64_t* total_entries, int64_t* total_rows, int32_t* max_rows,
                             void* stream) {
    int rc = check_gathers(d, true);
    if (rc) return rc;
    if (!central || n_central < 1) return fail(SEIS_EINVAL, "central must be non-NULL, n >= 1");
    if (!(apm >= 0.f)) return fail(SEIS_EINVAL, "apm must be >= 0");
    if (!(hmax >= 0.f)) return fail(SEIS_EINVAL, "hmax must be >= 0");
    if (!nbr_off || !m_c || !out_off || !dt_c) return fail(SEIS_EINVAL, "an output array is NULL");
    if (n_central > INT32_MAX) return fail(SEIS_EINVAL, "too many centrals");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = n_central;
    cudaError_t e;
    // counts -> nbr_off[1..n], rows -> out_off[1..n], prefix sums on the host.
    aperture_count_kernel<<<(unsigned)n, 256, 0, s>>>(d->midpoint, d->half_offset, d->gather_off,
                                                      d->out_off, d->dt, d->ngathers, d->ntraces,
                                                      central, apm, hmax, nbr_off + 1, m_c,
                                                      out_off + 1, dt_c);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "aperture count");
    std::vector<int64_t> cnt(n + 1), rows(n + 1);
    e = cudaMemcpyAsync(cnt.data() + 1, nbr_off + 1, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rows.data() + 1, out_off + 1, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "seis_crs_aperture");
    for (int64_t c = 1; c <= n; ++c)
        if (cnt[c] < 0) return fail(SEIS_EINVAL, "central %lld: gather index out of range or empty", (long long)(c - 1));
    cnt[0] = 0;
    rows[0] = 0;
    int64_t mr = 0;
    for (int64_t c = 0; c < n; ++c) {
        if (rows[c + 1] > mr) mr = rows[c + 1];
        cnt[c + 1] += cnt[c];
        rows[c + 1] += rows[c];
    }
    e = cudaMemcpyAsync(nbr_off, cnt.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_off, rows.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "seis_crs_aperture");
    if (total_entries) *total_entries = cnt[n];
    if (total_rows) *total_rows = rows[n];
    if (max_rows) *max_rows = (int32_t)mr;
    if (nbr_trace) {
        if (capacity < cnt[n]) {
            cudaStreamSynchronize(s);
            return fail(SEIS_EINVAL, "nbr_trace capacity %lld < %lld entries", (long long)capacity,
                        (long long)cnt[n]);
        }
        aperture_fill_kernel<<<(unsigned)n, 256, 0, s>>>(d->midpoint, d->half_offset, d->ntraces,
                                                         nbr_off, m_c, apm, hmax, nbr_trace);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "aperture fill");
    }
    e = cudaStreamSynchronize(s);   // host vectors above are released on return
    if (e != cudaSuccess) return cuda_fail(e, "seis_crs_aperture");
    return SEIS_OK;
}

extern "C" int seis_crs_aperture(const seis_gathers* d, const int32_t* central, int64_t n_central,
                                 float apm, int64_t* nbr_off, int32_t* nbr_trace, int64_t capacity,
                                 float* m_c, int64_t* out_off, float* dt_c, int64_t* total_entries,
                                 int64_t* total_rows, int32_t* max_rows, void* stream) {
    return crs_aperture_impl(d, central, n_central, apm, INFINITY, nbr_off, nbr_trace, capacity,
                             m_c, out_off, dt_c, total_entries, total_rows, max_rows, stream);
}

extern "C" int seis_crs_aperture_offset(const seis_gathers* d, const int32_t* central,
                                        int64_t n_central, float apm, float hmax,
                                        int64_t* nbr_off, int32_t* nbr_trace, int64_t capacity,
                                        float* m_c, int64_t* out_off, float* dt_c,
                                        int64_t* total_entries, int64_t* total_rows,
                                        int32_t* max_rows, void* stream) {
    return crs_aperture_impl(d, central, n_central, apm, hmax, nbr_off, nbr_trace, capacity,
                             m_c, out_off, dt_c, total_entries, total_rows, max_rows, stream);
}

// ------------------------------------------------------------------ wait self-test ----
namespace seis {

// One thread waits on a shared-memory mbarrier whose phase never completes (its single
// expected arrival never comes), through the same bounded wait the kernels use.
__global__ void selftest_wait_kernel(unsigned long long limit_ns, unsigned* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!mbar_wait_bounded(&bar, 0u, limit_ns)) record_status(status, kStatusTimeout);
    }
}

}  // namespace seis

extern "C" int seis_selftest_wait_timeout(int32_t limit_us, void* stream) {
    if (limit_us < 1 || limit_us > 1000000) return fail(SEIS_EINVAL, "limit_us outside [1, 1e6]");
    selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        (unsigned long long)limit_us * 1000ull, device_status_word());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "seis_selftest_wait_timeout");
    return SEIS_OK;
}
