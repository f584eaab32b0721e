// search_kernel.cuh -- the semblance search kernel (CMP and CRS) for sm_103a.
//
// What it computes (arXiv:1907.11678): Section 2.1 / Eq. 1 (windowed semblance with the
// 1/N normalisation), Algorithm 1 (per (t0, candidate) pair: intersect every trace,
// interpolate v = (c[j+1]-c[j])*x + c[j] along the window, accumulate num[j], den and the
// linear stack), Section 3.2 (argmax over candidates, stack at the pick), and for CRS
// Section 2.2 / 3.5 (the aperture's traces and the A/B/C traveltime surface).
//
// How (GB300 design; the paper's Algorithm 2 "re-design" idea of reusing one staged
// trace window for many (t0, candidate) pairs, realised with the TMA engine):
//   - one CTA = one owner (CMP gather or CRS central CDP) x 32 consecutive output rows;
//     lane l of every warp owns row n0 + l, so the 32 lanes of a warp read 32 nearby
//     sample indices of the same trace (no bank conflicts, often broadcasts);
//   - candidates are processed in passes of 32: each thread keeps the accumulators of 4
//     candidates (num[w], den, N) in registers for the whole trace loop;
//   - per pass, traces stream through a double-buffered shared-memory ring in stages of
//     up to 64 traces: warp 0 computes, for every trace, the exact sample window that the
//     stage's 32 rows x 32 candidates can touch (traveltime bounds at the box corners,
//     +-2 samples of margin), and copies it with one 1-D bulk copy (cp.async.bulk) plus
//     at most 3+3 scalar edge loads; completion is tracked by an mbarrier transaction
//     count, so the next stage loads while the current one computes;
//   - the traveltime is formed in sample units as u = n + D with the cancellation-free
//     moveout D = C q / (sqrt(n^2 + C q) + n), q = (h/dt)^2, which keeps the
//     interpolation fraction accurate to ~1e-4 samples in FP32;
//   - the argmax over all candidates stays inside the CTA (register running best per
//     thread, then an 8-way shared-memory reduction), so no atomics and no cube.
#pragma once
#include <cfloat>
#include <climits>
#include "seis_dev.cuh"
#include "seis_internal.h"

namespace seis {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kR = 4;                  // candidates per thread per pass
constexpr int kCB = kWarps * kR;       // candidates per pass (= 32: one per planner lane)
constexpr int kChunkT = 64;            // traces per stage at most
constexpr int kBuf = 12288;            // floats per stage buffer (48 KB)
constexpr unsigned kFull = 0xffffffffu;

struct __align__(16) TraceMeta {
    int base;     // shared-memory float index of sample 0 of the trace in this stage's buffer
    int kmin;     // intersections with kmin <= k <= kmax take part (window inside trace,
    int kmax;     //   and inside the staged sample window)
    float q;      // (h/dt)^2
    float e;      // dm/dt            (CRS)
    float g;      // (dm/dt)^2        (CRS)
    int pad0, pad1;
};

struct __align__(16) StageDesc {
    int pass, ntr, first, last, end, pad0, pad1, pad2;
};

struct SearchSmem {
    float buf[2][kBuf];
    TraceMeta meta[2][kChunkT];
    StageDesc desc[2];
    uint64_t full[2];
    int abort_flag;
    int pad[3];
    float redS[kWarps][32];
    int redC[kWarps][32];
    float redT[kWarps][32];
};

__device__ __forceinline__ float warp_min(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

template <bool CRS>
__device__ __forceinline__ void decode_candidate(const SearchParams& P, int c, float& a, float& b,
                                                 float& cc) {
    if (CRS) {
        const int nbc = P.nB * P.nC;
        const int ia = c / nbc;
        const int rem = c - ia * nbc;
        const int ib = rem / P.nC;
        const int ic = rem - ib * P.nC;
        a = P.A[ia];
        b = P.B[ib];
        cc = P.C[ic];
    } else {
        a = 0.f;
        b = 0.f;
        cc = P.C[c];
    }
}

template <bool CRS, int W>
__global__ void __launch_bounds__(kThreads, 2) search_kernel(const SearchParams P) {
    constexpr int HW = W / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SearchSmem& sm = *reinterpret_cast<SearchSmem*>(smem_raw);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t owner = blockIdx.x / P.tiles_per_owner;
    const int tile = (int)(blockIdx.x - owner * P.tiles_per_owner);
    if (owner >= P.nowner) return;
    const int64_t row0 = P.out_off[owner];
    const int nrows = (int)(P.out_off[owner + 1] - row0);
    const int n0 = tile * 32;
    if (n0 >= nrows) return;                          // whole CTA: uniform
    const int64_t lbeg = P.list_off[owner];
    const int64_t M64 = P.list_off[owner + 1] - lbeg;
    const int M = M64 < 0 ? 0 : (M64 > INT_MAX ? INT_MAX : (int)M64);
    const float dt = P.dt[owner];
    const float mc = CRS ? P.m_c[owner] : 0.f;
    const int npass = (P.ncand + kCB - 1) / kCB;
    const int n = n0 + lane;
    const bool act = n < nrows;
    const int n_last = min(n0 + 31, nrows - 1);

    if (threadIdx.x == 0) {
        mbar_init(&sm.full[0], 32);
        mbar_init(&sm.full[1], 32);
        sm.abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // ---------------- planner (warp 0): stage sequence = passes x trace chunks ----------
    int pl_pass = 0, pl_t = 0, pl_bpass = -1;
    float bA0 = 0.f, bA1 = 0.f, bB0 = 0.f, bB1 = 0.f, bC0 = 0.f, bC1 = 0.f;

    auto plan = [&](int slot) {
        if (pl_pass >= npass) {
            if (lane == 0) sm.desc[slot] = StageDesc{0, 0, 0, 0, 1, 0, 0, 0};
            __syncwarp();
            mbar_arrive(&sm.full[slot]);
            return;
        }
        if (pl_bpass != pl_pass) {   // candidate bounds of this pass (one candidate per lane)
            const int c = pl_pass * kCB + lane;
            float a = 0.f, b = 0.f, cc = 0.f;
            const bool v = c < P.ncand;
            if (v) decode_candidate<CRS>(P, c, a, b, cc);
            bA0 = warp_min(v ? a : FLT_MAX);  bA1 = warp_max(v ? a : -FLT_MAX);
            bB0 = warp_min(v ? b : FLT_MAX);  bB1 = warp_max(v ? b : -FLT_MAX);
            bC0 = warp_min(v ? cc : FLT_MAX); bC1 = warp_max(v ? cc : -FLT_MAX);
            pl_bpass = pl_pass;
        }
        float* slotbuf = sm.buf[slot];
        const int first = (pl_t == 0);
        int cnt = 0, used = 0;
        fence_proxy_async_smem();    // earlier generic accesses of this slot before async writes
        while (cnt < kChunkT && pl_t < M) {
            const int t = pl_t + lane;
            const bool v = (t < M) && (cnt + lane < kChunkT);
            int len = 0, n_el = 0, mis = 0, lo = 0;
            const float* src = nullptr;
            TraceMeta tm{0, 1, 0, 0.f, 0.f, 0.f, 0, 0};
            if (v) {
                const int64_t tid = P.list ? (int64_t)P.list[lbeg + t] : (lbeg + t);
                const int64_t toff = P.trace_off[tid];
                const int64_t ns64 = P.trace_off[tid + 1] - toff;
                const int ns_i = ns64 < 0 ? 0 : (ns64 > (INT_MAX / 4) ? (INT_MAX / 4) : (int)ns64);
                const double dtd = (double)dt;
                const double hd = (double)P.h[tid];
                tm.q = (float)(hd * hd / (dtd * dtd));
                float aLo = 0.f, aHi = 0.f, rLo, rHi;
                if (CRS) {
                    const double dm = (double)P.m[tid] - (double)mc;
                    tm.e = (float)(dm / dtd);
                    tm.g = (float)(dm * dm / (dtd * dtd));
                    aLo = fminf(bA0 * tm.e, bA1 * tm.e);
                    aHi = fmaxf(bA0 * tm.e, bA1 * tm.e);
                    rLo = bB0 * tm.g + bC0 * tm.q;
                    rHi = bB1 * tm.g + bC1 * tm.q;
                } else {
                    rLo = bC0 * tm.q;
                    rHi = bC1 * tm.q;
                }
                const float pLo = fmaxf((float)n0 + aLo, 0.f);
                const float pHi = (float)n_last + aHi;
                const float radLo = pLo * pLo + rLo;
                const float radHi = pHi * pHi + rHi;
                if (pHi >= 0.f && radHi >= 0.f) {
                    const float uLo = fminf(sqrtf(fmaxf(radLo, 0.f)), 1.6e7f);
                    const float uHi = fminf(sqrtf(radHi), 1.6e7f);
                    const int klo = (int)floorf(uLo) - 2;
                    const int khi = (int)floorf(uHi) + 2;
                    const int kmin = max(klo, HW);
                    const int kmax = min(khi, ns_i - HW - 2);
                    if (kmin <= kmax) {
                        tm.kmin = kmin;
                        tm.kmax = kmax;
                        lo = kmin - HW;
                        n_el = (kmax + HW + 1) - lo + 1;
                        src = P.traces + toff + lo;
                        mis = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
                        len = (mis + n_el + 3) & ~3;
                    }
                }
            }
            int pre = len;                                       // inclusive scan of lengths
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, pre, o);
                if (lane >= o) pre += y;
            }
            const bool fits = v && (used + pre <= kBuf);
            const int nfit = __popc(__ballot_sync(kFull, fits));  // a prefix of the lanes
            if (nfit == 0) {
                if (cnt == 0) {      // a single window larger than the buffer: drop + flag
                    if (lane == 0) {
                        record_status(P.status, kStatusOverflow);
                        sm.meta[slot][0] = TraceMeta{0, 1, 0, 0.f, 0.f, 0.f, 0, 0};
                    }
                    cnt = 1;
                    pl_t += 1;
                    continue;
                }
                break;
            }
            if (lane < nfit) {
                const int off = used + pre - len;                  // multiple of 4 floats
                tm.base = off + mis - lo;
                sm.meta[slot][cnt + lane] = tm;
                if (n_el > 0) {
                    float* dst = slotbuf + off + mis;
                    const int head = min((4 - mis) & 3, n_el);
                    const int nb = (n_el - head) & ~3;
                    for (int e2 = 0; e2 < head; ++e2) dst[e2] = ldg_nc(src + e2);
                    for (int e2 = head + nb; e2 < n_el; ++e2) dst[e2] = ldg_nc(src + e2);
                    if (nb > 0) {
                        mbar_expect_tx(&sm.full[slot], (uint32_t)nb * 4u);
                        bulk_g2s(dst + head, src + head, (uint32_t)nb * 4u, &sm.full[slot]);
                    }
                }
            }
            used += __shfl_sync(kFull, pre, nfit - 1);
            cnt += nfit;
            pl_t += nfit;
        }
        const int last = (pl_t >= M);
        if (lane == 0) sm.desc[slot] = StageDesc{pl_pass, cnt, first, last, 0, 0, 0, 0};
        if (last) { ++pl_pass; pl_t = 0; }
        __syncwarp();
        mbar_arrive(&sm.full[slot]);
    };

    // ---------------- consumers (all warps) -------------------------------------------
    float num[kR][W];
    float den[kR];
    int cntv[kR];
    float Ar[kR], Br[kR], Cr[kR];
    int cidx[kR];
    float bestS = -1.f, bestT = 0.f;
    int bestC = INT_MAX;
    const float nf = (float)n;
    const float n2 = nf * nf;

    if (warp == 0) { plan(0); plan(1); }

    int it = 0;
    for (;; ++it) {
        const int slot = it & 1;
        if (!sm.abort_flag) {
            if (!mbar_wait_bounded(&sm.full[slot], (uint32_t)((it >> 1) & 1))) {
                sm.abort_flag = 1;
                record_status(P.status, kStatusTimeout);
            }
        }
        const StageDesc d = sm.desc[slot];
        if (d.end) break;
        if (d.first) {
            #pragma unroll
            for (int r = 0; r < kR; ++r) {
                const int c = d.pass * kCB + r * kWarps + warp;
                cidx[r] = c;
                Ar[r] = Br[r] = Cr[r] = 0.f;
                if (c < P.ncand) decode_candidate<CRS>(P, c, Ar[r], Br[r], Cr[r]);
                den[r] = 0.f;
                cntv[r] = 0;
                #pragma unroll
                for (int j = 0; j < W; ++j) num[r][j] = 0.f;
            }
        }
        const float* sbuf = sm.buf[slot];
        const int ntr = min(d.ntr, kChunkT);
        for (int t = 0; t < ntr; ++t) {
            const TraceMeta tm = sm.meta[slot][t];
            const float* fb = sbuf + (tm.base - HW);
            #pragma unroll
            for (int r = 0; r < kR; ++r) {
                if (cidx[r] >= P.ncand) continue;                  // warp-uniform
                float D;
                bool ok;
                if (CRS) {
                    const float a = Ar[r] * tm.e;
                    const float p = nf + a;
                    const float rr = fmaf(Br[r], tm.g, Cr[r] * tm.q);
                    const float rad = fmaf(p, p, rr);
                    const float s = sqrt_fast(rad);
                    D = fmaf(rr, rcp_fast(fmaxf(s + p, 1e-30f)), a);
                    ok = act && (p >= 0.f) && (rad >= 0.f);
                } else {
                    const float cq = Cr[r] * tm.q;
                    const float rad = n2 + cq;
                    const float s = sqrt_fast(rad);
                    D = cq * rcp_fast(fmaxf(s + nf, 1e-30f));
                    ok = act && (rad >= 0.f);
                }
                const float fl = floorf(D);
                const float x = D - fl;
                const int k = n + __float2int_rz(fminf(fl, 16777216.f));
                ok = ok && (k >= tm.kmin) && (k <= tm.kmax);
                if (ok) {
                    const float* p = fb + k;
                    float f[W + 1];
                    #pragma unroll
                    for (int j = 0; j <= W; ++j) f[j] = p[j];
                    #pragma unroll
                    for (int j = 0; j < W; ++j) {
                        const float v = fmaf(x, f[j + 1] - f[j], f[j]);
                        num[r][j] += v;
                        den[r] = fmaf(v, v, den[r]);
                    }
                    cntv[r] += 1;
                }
            }
        }
        if (d.last) {
            #pragma unroll
            for (int r = 0; r < kR; ++r) {
                const int c = cidx[r];
                if (c >= P.ncand) continue;
                float nu = 0.f, ac = 0.f;
                #pragma unroll
                for (int j = 0; j < W; ++j) { nu = fmaf(num[r][j], num[r][j], nu); ac += num[r][j]; }
                const float Nf = (float)cntv[r];
                const float s = (cntv[r] > 0 && den[r] > 0.f) ? nu / (Nf * den[r]) : 0.f;
                const float st = cntv[r] > 0 ? ac / (Nf * (float)W) : 0.f;
                if (P.S_cube && act) P.S_cube[(row0 + n) * (int64_t)P.ncand + c] = s;
                if (s > bestS) { bestS = s; bestC = c; bestT = st; }
            }
        }
        __syncthreads();                         // every consumer is done with this slot
        if (sm.abort_flag) break;
        if (warp == 0) plan(slot);
    }

    if (sm.abort_flag) {
        // Stages `it` and `it + 1` may still have copies in flight: let them land (bounded)
        // before the CTA's shared memory is released.
        if (threadIdx.x == 0) {
            mbar_wait_bounded(&sm.full[it & 1], (uint32_t)((it >> 1) & 1));
            mbar_wait_bounded(&sm.full[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        return;
    }

    sm.redS[warp][lane] = bestS;
    sm.redC[warp][lane] = bestC;
    sm.redT[warp][lane] = bestT;
    __syncthreads();
    if (warp == 0 && act) {
        float bs = sm.redS[0][lane], bt = sm.redT[0][lane];
        int bc = sm.redC[0][lane];
        #pragma unroll
        for (int w2 = 1; w2 < kWarps; ++w2) {
            const float s = sm.redS[w2][lane];
            const int c = sm.redC[w2][lane];
            if (s > bs || (s == bs && c < bc)) { bs = s; bc = c; bt = sm.redT[w2][lane]; }
        }
        if (bc == INT_MAX) { bc = 0; bs = 0.f; bt = 0.f; }
        const int64_t row = row0 + n;
        P.best_idx[row] = bc;
        P.best_S[row] = bs;
        P.stack[row] = bt;
        if (P.best_param) {
            float a, b, cc;
            decode_candidate<CRS>(P, bc, a, b, cc);
            if (CRS) {
                P.best_param[row * 3 + 0] = a;
                P.best_param[row * 3 + 1] = b;
                P.best_param[row * 3 + 2] = cc;
            } else {
                P.best_param[row] = cc;
            }
        }
    }
}

template <bool CRS, int W>
cudaError_t launch_search_w(const SearchParams& p, cudaStream_t stream) {
    static bool configured[64] = {};  // dynamic shared-memory opt-in, once per device
    const int smem = (int)sizeof(SearchSmem);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(search_kernel<CRS, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    const int64_t grid = p.nowner * (int64_t)p.tiles_per_owner;
    if (grid <= 0) return cudaSuccess;
    if (grid > INT_MAX) return cudaErrorInvalidValue;
    search_kernel<CRS, W><<<(unsigned)grid, kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

template <bool CRS>
cudaError_t launch_search_dispatch(const SearchParams& p, int w, cudaStream_t stream) {
    switch (w) {
        case 1: return launch_search_w<CRS, 1>(p, stream);
        case 3: return launch_search_w<CRS, 3>(p, stream);
        case 5: return launch_search_w<CRS, 5>(p, stream);
        case 7: return launch_search_w<CRS, 7>(p, stream);
        case 9: return launch_search_w<CRS, 9>(p, stream);
        case 11: return launch_search_w<CRS, 11>(p, stream);
        case 13: return launch_search_w<CRS, 13>(p, stream);
        case 15: return launch_search_w<CRS, 15>(p, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace seis
