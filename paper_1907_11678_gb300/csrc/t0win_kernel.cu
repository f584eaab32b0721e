// t0win_kernel.cu -- CMP and CRS semblance with the window over neighbouring output times
// (cmp_semblance_t0win, crs_semblance_t0win).  Not the paper's method: Algorithm 1 reads w samples along each
// trace around its own intersection, so every (row, candidate, trace) costs w
// interpolations; here the window runs over the output times t0' = t0 + j dt, each with its
// own traveltime (Section 2.1), so every (row, candidate, trace) costs one interpolation and
// the w-sample window is formed from the per-row sums of neighbouring rows:
//   s(t0') = sum_i v_i(t0'),  e(t0') = sum_i v_i(t0')^2,  M(t0') = traces taking part
//   (k >= 0 and k + 1 <= ns - 1),  S(t0) = sum_j s(t0')^2 / sum_j M(t0') e(t0'),
//   stack(t0) = s(t0) / M(t0) at the pick.
//
// Same CTA structure as the search kernel (producer warp staging trace windows through the
// shared-memory ring, consumer warps = candidates, lanes = rows), with a block of 64
// consecutive output times per CTA: lane l holds positions l and l + 32 as one f32x2 pair
// (the traveltime and interpolation of both run in packed FP32), the 64 - 2 hw middle
// positions are output rows, and each forms the window sums of its neighbours by warp
// shuffles.
#include "search_kernel.cuh"

namespace seis {

namespace {

constexpr int kTwWarps = 15;          // consumer warps
constexpr int kTwR = 2;               // candidates per thread
constexpr int kTwCB = kTwWarps * kTwR;
static_assert(kTwCB <= 32, "the producer bounds one candidate per lane");
static_assert(kTwWarps <= kMaxWarps, "reduction arrays are sized for kMaxWarps");
constexpr int kTwThreads = 32 * (kTwWarps + 1);

// Per thread: kTwR candidates at the lane's two output times (f32x2: .lo = row p0,
// .hi = row p0 + 32).
struct TwAccum {
    f2_t s2[kTwR], e2[kTwR];
    int M0[kTwR], M1[kTwR];
    float Ar[kTwR], Br[kTwR], Cr[kTwR];    // CMP: A = B = 0
    int cidx[kTwR];
};

struct TwRows {
    f2_t nf2, nsq2;      // (n0, n1) and their squares; inactive rows carry 2^24
    int n0, n1;
};

// One interpolated sample per (row pair, candidate, trace) of a run of traces [t0, t1):
// the moveout pair in samples, D = Cq / (sqrt(n^2 + Cq) + n) (CMP) or
// D = a + r / (sqrt(p^2 + r) + p) with a = A e, p = n + a, r = B g + C q (CRS), in f32x2,
// floor and fraction by the rounding shift, then v = f[k] + x (f[k+1] - f[k]).  The
// traveltimes of trace t+1 are formed while trace t is interpolated.
template <bool CRS, bool FAST>
__device__ __forceinline__ void tw_run(TwAccum& a, const TraceMeta* meta, int t0, int t1,
                                       const TwRows& rw, int zidx, const float* smf) {
    int sI0[kTwR], sI1[kTwR];
    f2_t sX2[kTwR];
    bool sO0[kTwR], sO1[kTwR];
    const f2_t shift2 = pk2(kFloorShift, kFloorShift);
    auto setup = [&](int t) {
        const TraceMeta& tm = meta[t];
        const unsigned rng = tm.rng;
        const int kbase = tm.kbase;
        const int off0 = rw.n0 + tm.offk;
        const int off1 = rw.n1 + tm.offk;
        #pragma unroll
        for (int r = 0; r < kTwR; ++r) {
            f2_t D2;
            bool p0 = true, p1 = true;
            if constexpr (CRS) {
                const float av = a.Ar[r] * tm.e;
                const float rr = fmaf(a.Br[r], tm.g, a.Cr[r] * tm.q);
                const f2_t a2 = pk2(av, av), rr2 = pk2(rr, rr);
                const f2_t pp2 = add2(rw.nf2, a2);
                const f2_t rad2 = fma2(pp2, pp2, rr2);
                float ra, rb, pa, pb;
                up2(rad2, ra, rb);
                up2(pp2, pa, pb);
                p0 = pa >= 0.f;
                p1 = pb >= 0.f;
                const f2_t sum2 = add2(pk2(sqrt_fast(ra), sqrt_fast(rb)), pp2);
                float sa, sb;
                up2(sum2, sa, sb);
                if constexpr (!FAST) { sa = fmaxf(sa, 1e-30f); sb = fmaxf(sb, 1e-30f); }
                D2 = fma2(rr2, pk2(rcp_fast(sa), rcp_fast(sb)), a2);
            } else {
                const float cq = a.Cr[r] * tm.q;
                const f2_t cq2 = pk2(cq, cq);
                const f2_t rad2 = add2(rw.nsq2, cq2);
                float ra, rb;
                up2(rad2, ra, rb);
                const f2_t sum2 = add2(pk2(sqrt_fast(ra), sqrt_fast(rb)), rw.nf2);
                float sa, sb;
                up2(sum2, sa, sb);
                D2 = mul2(cq2, pk2(rcp_fast(sa), rcp_fast(sb)));
            }
            const f2_t tt2 = add2_rm(D2, shift2);
            f2_t x2 = sub2(D2, sub2(tt2, shift2));
            float ta, tb;
            up2(tt2, ta, tb);
            const int kk0 = __float_as_int(ta) + off0;
            const int kk1 = __float_as_int(tb) + off1;
            if constexpr (FAST) {
                sI0[r] = kbase + (int)min((unsigned)kk0, rng);
                sI1[r] = kbase + (int)min((unsigned)kk1, rng);
                sO0[r] = sO1[r] = true;
            } else {
                const bool ok0 = p0 && (unsigned)kk0 <= rng, ok1 = p1 && (unsigned)kk1 <= rng;
                float xa, xb;
                up2(x2, xa, xb);
                x2 = pk2(ok0 ? xa : 0.f, ok1 ? xb : 0.f);   // a NaN fraction must not reach the sums
                sI0[r] = ok0 ? kbase + kk0 : zidx;
                sI1[r] = ok1 ? kbase + kk1 : zidx;
                sO0[r] = ok0;
                sO1[r] = ok1;
            }
            sX2[r] = x2;
        }
    };
    setup(t0);
    auto step = [&](int t, auto more) {
        int cI0[kTwR], cI1[kTwR];
        f2_t cX2[kTwR];
        #pragma unroll
        for (int r = 0; r < kTwR; ++r) {
            cI0[r] = sI0[r];
            cI1[r] = sI1[r];
            cX2[r] = sX2[r];
            a.M0[r] += sO0[r] ? 1 : 0;
            a.M1[r] += sO1[r] ? 1 : 0;
        }
        if constexpr (decltype(more)::value) setup(t + 1);
        #pragma unroll
        for (int r = 0; r < kTwR; ++r) {
            const f2_t f0 = pk2(smf[cI0[r]], smf[cI1[r]]);
            const f2_t f1 = pk2(smf[cI0[r] + 1], smf[cI1[r] + 1]);
            const f2_t v2 = fma2(cX2[r], sub2(f1, f0), f0);
            a.s2[r] = add2(a.s2[r], v2);
            a.e2[r] = fma2(v2, v2, a.e2[r]);
        }
    };
    for (int t = t0; t < t1 - 1; ++t) step(t, std::true_type{});
    step(t1 - 1, std::false_type{});           // the run's last trace sets up nothing
}

// Window sums of the output time at position p = lane + 32 h (h = 0, 1) of the 64-row
// block: positions p + j, j = -hw..hw, inside [0, 64).  Position q < 32 is lane q's .lo
// value, q >= 32 is lane q - 32's .hi value.
template <int HW>
__device__ __forceinline__ void window_sums2(float s_lo, float s_hi, float m_lo, float m_hi,
                                             int lane, float& num0, float& den0, float& num1,
                                             float& den1) {
    num0 = den0 = num1 = den1 = 0.f;
    #pragma unroll
    for (int j = -HW; j <= HW; ++j) {
        const int src = (lane + j) & 31;
        const float sa = __shfl_sync(kFull, s_lo, src), sb = __shfl_sync(kFull, s_hi, src);
        const float ma = __shfl_sync(kFull, m_lo, src), mb = __shfl_sync(kFull, m_hi, src);
        const int q = lane + j;                     // position of row 0's neighbour
        // row 0 (position lane): q < 0 outside, q < 32 a lo value, else a hi value
        if (q >= 0) {
            const float sv = q < 32 ? sa : sb, mv = q < 32 ? ma : mb;
            num0 = fmaf(sv, sv, num0);
            den0 += mv;
        }
        // row 1 (position 32 + lane): q < 0 a lo value, q < 32 a hi value, else outside
        if (q < 32) {
            const float sv = q < 0 ? sa : sb, mv = q < 0 ? ma : mb;
            num1 = fmaf(sv, sv, num1);
            den1 += mv;
        }
    }
}

template <bool CRS, int W>
__global__ void __launch_bounds__(kTwThreads, 2) t0win_kernel(const SearchParams P) {
    constexpr int HW = W / 2;
    constexpr int kT = 64 - 2 * HW;              // output rows per CTA
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SearchSmem& sm = *reinterpret_cast<SearchSmem*>(smem_raw);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t owner = blockIdx.x / P.tiles_per_owner;
    const int tile = (int)(blockIdx.x - owner * P.tiles_per_owner);
    if (owner >= P.nowner) return;
    const int64_t row0 = P.out_off[owner];
    const int nrows = (int)(P.out_off[owner + 1] - row0);
    const int first_out = tile * kT;              // first output row of the CTA
    if (first_out >= nrows) return;               // whole CTA: uniform
    const int base = first_out - HW;              // row of position 0
    const int64_t lbeg = P.list_off[owner];
    const int64_t M64 = P.list_off[owner + 1] - lbeg;
    const int M = M64 < 0 ? 0 : (M64 > INT_MAX ? INT_MAX : (int)M64);
    const float dt = P.dt[owner];
    const int npass = (P.ncand + kTwCB - 1) / kTwCB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&sm.full[s], 32);
            mbar_init(&sm.empty[s], 32 * kTwWarps);
        }
        sm.abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 16) sm.zeros[threadIdx.x] = 0.f;
    __syncthreads();

    if (warp == kTwWarps) {
        // =============================== producer warp ================================
        const int n_first = max(base, 0);
        const int n_last = min(base + 63, nrows - 1);
        const float mc = CRS ? P.m_c[owner] : 0.f;
        int pl_pass = 0, pl_t = 0, pl_bpass = -1;
        float bA0 = 0.f, bA1 = 0.f, bB0 = 0.f, bB1 = 0.f, bC0 = 0.f, bC1 = 0.f;
        int s = 0;
        for (;; ++s) {
            const int slot = s % kSlots;
            if (s >= kSlots && !sm.abort_flag) {
                if (!mbar_wait_backoff(&sm.empty[slot], (uint32_t)(((s / kSlots) & 1) ^ 1))) {
                    sm.abort_flag = 1;
                    record_status(P.status, kStatusTimeout);
                }
            }
            __syncwarp();
            if (sm.abort_flag || pl_pass >= npass) {
                if (lane == 0) sm.desc[slot] = make_desc(0, 0, 0u, 0, 0, 1);
                __syncwarp();
                mbar_arrive(&sm.full[slot]);
                break;
            }
            if (pl_bpass != pl_pass) {   // candidate bounds of the pass (one per lane)
                const int c = pl_pass * kTwCB + lane;
                const bool v = lane < kTwCB && c < P.ncand;
                float av = 0.f, bv = 0.f, cc = 0.f;
                if (v) decode_candidate<CRS>(P, c, av, bv, cc);
                bA0 = warp_min(v ? av : FLT_MAX);  bA1 = warp_max(v ? av : -FLT_MAX);
                bB0 = warp_min(v ? bv : FLT_MAX);  bB1 = warp_max(v ? bv : -FLT_MAX);
                bC0 = warp_min(v ? cc : FLT_MAX);  bC1 = warp_max(v ? cc : -FLT_MAX);
                pl_bpass = pl_pass;
            }
            const int first = (pl_t == 0);
            int nfit = 0;
            unsigned allv = 0u;
            const int ntr = produce_stage<CRS, 0>(
                sm.buf[slot], (int)(sm.buf[slot] - reinterpret_cast<float*>(smem_raw)),
                sm.meta[slot], &sm.full[slot], P.traces, P.trace_off, P.h,
                CRS ? P.m : nullptr, P.list, lbeg, M, pl_t, dt, mc, n_first, n_last,
                StageBounds{bA0, bA1, bB0, bB1, bC0, bC1}, P.status, nfit, allv);
            pl_t += nfit;
            const int last = (pl_t >= M);
            if (lane == 0) sm.desc[slot] = make_desc(pl_pass, ntr, allv, first, last, 0);
            if (last) { ++pl_pass; pl_t = 0; }
            __syncwarp();
            mbar_arrive(&sm.full[slot]);
        }
        const int s_end = s;
        for (int s2 = max(0, s_end - kSlots + 1); s2 <= s_end; ++s2)
            mbar_wait_bounded(&sm.full[s2 % kSlots], (uint32_t)((s2 / kSlots) & 1));
        return;
    }

    // ================================ consumer warps =====================================
    const float* smf = reinterpret_cast<const float*>(smem_raw);
    const int zidx = (int)(reinterpret_cast<const float*>(sm.zeros) - smf);
    const int n0 = base + lane, n1 = base + 32 + lane;
    const bool act0 = n0 >= 0 && n0 < nrows, act1 = n1 < nrows;
    const bool is_out0 = act0 && lane >= HW;              // positions HW .. 63 - HW
    const bool is_out1 = act1 && 32 + lane < 64 - HW;
    TwRows rw;
    rw.n0 = act0 ? n0 : (1 << 24);
    rw.n1 = act1 ? n1 : (1 << 24);
    {
        const float f0 = fmaxf((float)rw.n0, 1e-30f), f1 = fmaxf((float)rw.n1, 1e-30f);
        rw.nf2 = pk2(f0, f1);
        rw.nsq2 = pk2(f0 * f0, f1 * f1);
    }
    TwAccum a;
    #pragma unroll
    for (int r = 0; r < kTwR; ++r) a.cidx[r] = INT_MAX;
    float bestS0 = -1.f, bestT0 = 0.f, bestS1 = -1.f, bestT1 = 0.f;
    int bestC0 = INT_MAX, bestC1 = INT_MAX;
    bool aborted = false;

    for (int s = 0;; ++s) {
        const int slot = s % kSlots;
        if (!mbar_wait_bounded(&sm.full[slot], (uint32_t)((s / kSlots) & 1))) {
            sm.abort_flag = 1;
            record_status(P.status, kStatusTimeout);
            aborted = true;
            break;
        }
        const StageDesc d = sm.desc[slot];
        if (d.end) {
            aborted = sm.abort_flag != 0;
            break;
        }
        if (d.first) {
            #pragma unroll
            for (int r = 0; r < kTwR; ++r) {
                const int c = d.pass * kTwCB + warp * kTwR + r;
                a.Ar[r] = a.Br[r] = a.Cr[r] = 0.f;
                if (c < P.ncand) decode_candidate<CRS>(P, c, a.Ar[r], a.Br[r], a.Cr[r]);
                a.cidx[r] = c;
                a.s2[r] = 0ull;
                a.e2[r] = 0ull;
                a.M0[r] = a.M1[r] = 0;
            }
        }
        const int ntr = min(d.ntr, kChunkT);
        if (ntr > 0 && a.cidx[0] < P.ncand) {
            int t = 0;
            while (t < ntr) {                          // runs of check-free / checked traces
                const bool fast = (d.allv >> t) & 1u;
                const unsigned rest = (fast ? ~d.allv : d.allv) >> t;
                const int len = rest ? __ffs(rest) - 1 : 32;
                const int t1 = min(ntr, t + len);
                if (fast) tw_run<CRS, true>(a, sm.meta[slot], t, t1, rw, zidx, smf);
                else tw_run<CRS, false>(a, sm.meta[slot], t, t1, rw, zidx, smf);
                t = t1;
            }
        }
        if (d.last) {
            #pragma unroll
            for (int r = 0; r < kTwR; ++r) {
                const int c = a.cidx[r];
                float s_lo, s_hi, e_lo, e_hi;
                up2(a.s2[r], s_lo, s_hi);
                up2(a.e2[r], e_lo, e_hi);
                // inactive rows contributed nothing: their s, e, M count as 0
                if (!act0) { s_lo = 0.f; e_lo = 0.f; }
                if (!act1) { s_hi = 0.f; e_hi = 0.f; }
                const float m_lo = act0 ? (float)a.M0[r] * e_lo : 0.f;
                const float m_hi = act1 ? (float)a.M1[r] * e_hi : 0.f;
                float num0, den0, num1, den1;
                window_sums2<HW>(s_lo, s_hi, m_lo, m_hi, lane, num0, den0, num1, den1);
                if (c >= P.ncand) continue;
                if (is_out0) {
                    const float sv = den0 > 0.f ? num0 / den0 : 0.f;
                    const float st = a.M0[r] > 0 ? s_lo / (float)a.M0[r] : 0.f;
                    if (P.S_cube) P.S_cube[(row0 + n0) * (int64_t)P.ncand + c] = sv;
                    if (sv > bestS0) { bestS0 = sv; bestC0 = c; bestT0 = st; }
                }
                if (is_out1) {
                    const float sv = den1 > 0.f ? num1 / den1 : 0.f;
                    const float st = a.M1[r] > 0 ? s_hi / (float)a.M1[r] : 0.f;
                    if (P.S_cube) P.S_cube[(row0 + n1) * (int64_t)P.ncand + c] = sv;
                    if (sv > bestS1) { bestS1 = sv; bestC1 = c; bestT1 = st; }
                }
            }
        }
        mbar_arrive(&sm.empty[slot]);
    }

    // two rounds of the cross-warp argmax: the lane's lower row, then its upper row
    for (int h = 0; h < 2; ++h) {
        sm.redS[warp][lane] = h ? bestS1 : bestS0;
        sm.redC[warp][lane] = h ? bestC1 : bestC0;
        sm.redT[warp][lane] = h ? bestT1 : bestT0;
        consumer_bar(32 * kTwWarps);
        const bool outh = h ? is_out1 : is_out0;
        if (!aborted && !sm.abort_flag && warp == 0 && outh) {
            float bs, bt;
            int bc;
            reduce_best(sm, kTwWarps, lane, bs, bc, bt);
            const int64_t row = row0 + (h ? n1 : n0);
            P.best_idx[row] = bc;
            P.best_S[row] = bs;
            P.stack[row] = bt;
            if (P.best_param) {
                float av, bv, cc;
                decode_candidate<CRS>(P, bc, av, bv, cc);
                if (CRS) {
                    P.best_param[row * 3 + 0] = av;
                    P.best_param[row * 3 + 1] = bv;
                    P.best_param[row * 3 + 2] = cc;
                } else {
                    P.best_param[row] = cc;
                }
            }
        }
        consumer_bar(32 * kTwWarps);                 // the arrays are reused
    }
}

template <bool CRS, int W>
cudaError_t launch_t0win_w(SearchParams p, int max_rows, cudaStream_t stream) {
    static bool configured[64] = {};
    const int smem = (int)sizeof(SearchSmem);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(t0win_kernel<CRS, W>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    constexpr int kT = 64 - 2 * (W / 2);
    p.tiles_per_owner = (max_rows + kT - 1) / kT;
    const int64_t grid = p.nowner * (int64_t)p.tiles_per_owner;
    if (grid <= 0) return cudaSuccess;
    if (grid > INT_MAX) return cudaErrorInvalidValue;
    t0win_kernel<CRS, W><<<(unsigned)grid, kTwThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

template <bool CRS>
cudaError_t launch_t0win_c(const SearchParams& p, int w, int max_rows, cudaStream_t s) {
    switch (w) {
        case 1: return launch_t0win_w<CRS, 1>(p, max_rows, s);
        case 3: return launch_t0win_w<CRS, 3>(p, max_rows, s);
        case 5: return launch_t0win_w<CRS, 5>(p, max_rows, s);
        case 7: return launch_t0win_w<CRS, 7>(p, max_rows, s);
        case 9: return launch_t0win_w<CRS, 9>(p, max_rows, s);
        case 11: return launch_t0win_w<CRS, 11>(p, max_rows, s);
        case 13: return launch_t0win_w<CRS, 13>(p, max_rows, s);
        case 15: return launch_t0win_w<CRS, 15>(p, max_rows, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace seis

using namespace seis;

extern "C" int cmp_semblance_t0win(const seis_gathers* d, const float* C, int32_t nc, int32_t w,
                                   float* S_cube, int32_t* best_idx, float* best_C,
                                   float* best_S, float* stack_out, void* stream) {
    SearchParams p;
    TuneKey key;
    int rc = build_cmp_params(d, C, nc, w, S_cube, best_idx, best_C, best_S, stack_out, &p, &key);
    if (rc) return rc;
    cudaError_t e = launch_t0win_c<false>(p, w, d->max_rows, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cmp_semblance_t0win launch");
    return SEIS_OK;
}

extern "C" int crs_semblance_t0win(const seis_gathers* d, const seis_aperture* ap,
                                   const float* A, int32_t nA, const float* B, int32_t nB,
                                   const float* C, int32_t nC, int32_t w, float* S_cube,
                                   int32_t* best_idx, float* best_ABC, float* best_S,
                                   float* stack_out, void* stream) {
    SearchParams p;
    TuneKey key;
    int rc = build_crs_params(d, ap, A, nA, B, nB, C, nC, w, S_cube, best_idx, best_ABC, best_S,
                              stack_out, &p, &key);
    if (rc) return rc;
    cudaError_t e = launch_t0win_c<true>(p, w, ap->max_rows, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "crs_semblance_t0win launch");
    return SEIS_OK;
}
