// seis_tune.cu -- the search-kernel autotuner: times every kernel variant on the caller's
// problem with CUDA events, keeps the fastest per shape bucket (in memory, savable as
// JSON), and answers the launch path's lookups.
#include <cuda_runtime.h>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>
#include "seis.h"
#include "seis_internal.h"

namespace seis {

static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tuned;

static int log2_bucket(int64_t v) {
    int b = 0;
    while (v > 1) { v >>= 1; ++b; }
    return b;
}

TuneKey make_tune_key(bool crs, int w, int ncand, int64_t max_rows, int64_t mean_fold) {
    return TuneKey{crs ? 1 : 0, w, log2_bucket(ncand), log2_bucket(max_rows), log2_bucket(mean_fold)};
}

int lookup_variant(const TuneKey& k, int fallback) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(k);
    return it == g_tuned.end() ? fallback : it->second;
}

void remember_variant(const TuneKey& k, int v) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[k] = v;
}

// Times each variant: one untimed launch, then `reps` launches between two events.
static int tune(SearchParams p, bool crs, int w, int reps, cudaStream_t s, const TuneKey& key,
                int* chosen, float* ms_out) {
    if (reps < 1) reps = 1;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(e, "autotune"); }
    int best = -1;
    float best_ms = 0.f;
    int rc = SEIS_OK;
    for (int v = 0; v < search_variant_count() && rc == SEIS_OK; ++v) {
        p.variant = v;
        float ms = 0.f;
        e = launch_search(p, crs, w, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_search(p, crs, w, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { rc = cuda_fail(e, "autotune launch"); break; }
        ms /= (float)reps;
        if (ms_out) ms_out[v] = ms;
        if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    remember_variant(key, best);
    if (chosen) *chosen = best;
    return SEIS_OK;
}

}  // namespace seis

using namespace seis;

extern "C" int seis_autotune_cmp(const seis_gathers* d, const float* C, int32_t nc, int32_t w,
                                 int32_t* best_idx, float* best_S, float* stack_out, int32_t reps,
                                 int32_t* chosen, float* ms_out, void* stream) {
    SearchParams p;
    TuneKey key;
    int rc = build_cmp_params(d, C, nc, w, nullptr, best_idx, nullptr, best_S, stack_out, &p, &key);
    if (rc) return rc;
    return tune(p, false, w, reps, static_cast<cudaStream_t>(stream), key, chosen, ms_out);
}

extern "C" int seis_autotune_crs(const seis_gathers* d, const seis_aperture* ap, const float* A,
                                 int32_t nA, const float* B, int32_t nB, const float* C,
                                 int32_t nC, int32_t w, int32_t* best_idx, float* best_S,
                                 float* stack_out, int32_t reps, int32_t* chosen, float* ms_out,
                                 void* stream) {
    SearchParams p;
    TuneKey key;
    int rc = build_crs_params(d, ap, A, nA, B, nB, C, nC, w, nullptr, best_idx, nullptr, best_S,
                              stack_out, &p, &key);
    if (rc) return rc;
    return tune(p, true, w, reps, static_cast<cudaStream_t>(stream), key, chosen, ms_out);
}

extern "C" int seis_autotune_save(const char* path) {
    if (!path) return fail(SEIS_EINVAL, "path is NULL");
    FILE* f = fopen(path, "w");
    if (!f) return fail(SEIS_EINVAL, "cannot write %s", path);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    fprintf(f, "{\"format\": \"seis-autotune-1\", \"entries\": [\n");
    size_t i = 0;
    for (const auto& kv : g_tuned) {
        const TuneKey& k = kv.first;
        fprintf(f, "  {\"crs\": %d, \"w\": %d, \"cand_bucket\": %d, \"rows_bucket\": %d, "
                   "\"fold_bucket\": %d, \"variant\": %d}%s\n",
                k.crs, k.w, k.cand_bucket, k.rows_bucket, k.fold_bucket, kv.second,
                ++i < g_tuned.size() ? "," : "");
    }
    fprintf(f, "]}\n");
    fclose(f);
    return SEIS_OK;
}

extern "C" int seis_autotune_load(const char* path) {
    if (!path) return fail(SEIS_EINVAL, "path is NULL");
    FILE* f = fopen(path, "r");
    if (!f) return fail(SEIS_EINVAL, "cannot read %s", path);
    std::vector<char> buf;
    char tmp[4096];
    size_t n;
    while ((n = fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
    fclose(f);
    buf.push_back('\0');
    // entries are flat objects with six integer fields written by seis_autotune_save
    int loaded = 0;
    const char* p = strstr(buf.data(), "\"entries\"");
    while (p && (p = strchr(p, '{')) != nullptr) {
        TuneKey k{};
        int v = -1;
        if (sscanf(p, "{\"crs\": %d, \"w\": %d, \"cand_bucket\": %d, \"rows_bucket\": %d, "
                      "\"fold_bucket\": %d, \"variant\": %d}",
                   &k.crs, &k.w, &k.cand_bucket, &k.rows_bucket, &k.fold_bucket, &v) != 6)
            return fail(SEIS_EINVAL, "malformed autotune entry in %s", path);
        if (v < 0 || v >= search_variant_count())
            return fail(SEIS_EINVAL, "variant %d out of range in %s", v, path);
        remember_variant(k, v);
        ++loaded;
        ++p;
    }
    return loaded >= 0 ? SEIS_OK : SEIS_EINVAL;
}

extern "C" int seis_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    return SEIS_OK;
}
