// t0win_kernel.cu -- CMP semblance with the window over neighbouring output times
// (cmp_semblance_t0win).  Not the paper's method: Algorithm 1 reads w samples along each
// trace around its own intersection, so every (row, candidate, trace) costs w
// interpolations; here the window runs over the output times t0' = t0 + j dt, each with its
// own traveltime (Section 2.1), so every (row, candidate, trace) costs one interpolation and
// the w-sample window is formed from the per-row sums of neighbouring rows:
//   s(t0') = sum_i v_i(t0'),  e(t0') = sum_i v_i(t0')^2,  M(t0') = traces taking part
//   (k >= 0 and k + 1 <= ns - 1),  S(t0) = sum_j s(t0')^2 / sum_j M(t0') e(t0'),
//   stack(t0) = s(t0) / M(t0) at the pick.
//
// Same CTA structure as the search kernel (producer warp staging trace windows through the
// shared-memory ring, consumer warps = candidates, lanes = rows), with lane l holding the
// output time n0 - hw + l: the 32 lanes compute s, e, M for 32 consecutive rows and the
// 32 - 2 hw middle lanes form the window sums of their neighbours by warp shuffles.
#include "search_kernel.cuh"

namespace seis {

namespace {

constexpr int kTwWarps = 13;          // consumer warps
constexpr int kTwR = 4;               // candidates per thread (independent traveltime chains)
constexpr int kTwCB = kTwWarps * kTwR;
static_assert(kTwCB <= 64, "the producer bounds two candidates per lane");
static_assert(kTwWarps <= kMaxWarps, "reduction arrays are sized for kMaxWarps");
constexpr int kTwThreads = 32 * (kTwWarps + 1);

struct TwAccum {
    float s[kTwR], e[kTwR];
    int M[kTwR];
    float Cr[kTwR];
    int cidx[kTwR];
};

// One interpolated sample per (row, candidate, trace) of a run of traces [t0, t1).  The
// traveltimes of trace t+1 (the MUFU chains) are formed while trace t is interpolated.
template <bool FAST>
__device__ __forceinline__ void tw_run(TwAccum& a, const TraceMeta* meta, int t0, int t1,
                                       int slot_base, const RowConst& rc, int zidx,
                                       const float* smf) {
    int sI[kTwR];
    float sX[kTwR];
    bool sO[kTwR];
    auto setup = [&](int t) {
        const TraceConst tc = trace_const(meta[t], rc.n, slot_base, 0);
        #pragma unroll
        for (int r = 0; r < kTwR; ++r) {
            if constexpr (FAST) {
                intersect_one_fast<false>(0.f, 0.f, a.Cr[r], tc, rc.nf, rc.nsq, sI[r], sX[r]);
                sO[r] = true;
            } else {
                intersect_one<false>(0.f, 0.f, a.Cr[r], tc, rc.nf, rc.nsq, zidx, sI[r], sX[r],
                                     sO[r]);
            }
        }
    };
    setup(t0);
    for (int t = t0; t < t1; ++t) {
        int cI[kTwR];
        float cX[kTwR];
        #pragma unroll
        for (int r = 0; r < kTwR; ++r) {
            cI[r] = sI[r];
            cX[r] = sX[r];
            a.M[r] += sO[r] ? 1 : 0;
        }
        setup(min(t + 1, t1 - 1));
        #pragma unroll
        for (int r = 0; r < kTwR; ++r) {
            const float f0 = smf[cI[r]], f1 = smf[cI[r] + 1];
            const float v = fmaf(cX[r], f1 - f0, f0);
            a.s[r] += v;
            a.e[r] = fmaf(v, v, a.e[r]);
        }
    }
}

// Sum over the lanes l + j, j = -hw..hw, that exist (lanes outside the warp give 0).
template <int HW>
__device__ __forceinline__ void window_sums(float s, float me, int lane, float& num, float& den) {
    num = 0.f;
    den = 0.f;
    #pragma unroll
    for (int j = -HW; j <= HW; ++j) {
        const int src = lane + j;
        const float sj = __shfl_sync(kFull, s, src & 31);
        const float mj = __shfl_sync(kFull, me, src & 31);
        const bool in = src >= 0 && src < 32;
        num = in ? fmaf(sj, sj, num) : num;
        den = in ? den + mj : den;
    }
}

template <int W>
__global__ void __launch_bounds__(kTwThreads, 2) t0win_kernel(const SearchParams P) {
    constexpr int HW = W / 2;
    constexpr int kT = 32 - 2 * HW;              // output rows per CTA
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SearchSmem& sm = *reinterpret_cast<SearchSmem*>(smem_raw);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t owner = blockIdx.x / P.tiles_per_owner;
    const int tile = (int)(blockIdx.x - owner * P.tiles_per_owner);
    if (owner >= P.nowner) return;
    const int64_t row0 = P.out_off[owner];
    const int nrows = (int)(P.out_off[owner + 1] - row0);
    const int out0 = tile * kT;                   // first output row of the CTA
    if (out0 >= nrows) return;                    // whole CTA: uniform
    const int lane_row0 = out0 - HW;              // row of lane 0
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
        const int n_first = max(lane_row0, 0);
        const int n_last = min(lane_row0 + 31, nrows - 1);
        int pl_pass = 0, pl_t = 0, pl_bpass = -1;
        float bC0 = 0.f, bC1 = 0.f;
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
            if (pl_bpass != pl_pass) {   // C bounds of the pass, up to 64 candidates
                float lo = FLT_MAX, hi = -FLT_MAX;
                #pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int cl = lane + 32 * k;
                    const int c = pl_pass * kTwCB + cl;
                    if (cl < kTwCB && c < P.ncand) {
                        const float cc = P.C[c];
                        lo = fminf(lo, cc);
                        hi = fmaxf(hi, cc);
                    }
                }
                bC0 = warp_min(lo);
                bC1 = warp_max(hi);
                pl_bpass = pl_pass;
            }
            const int first = (pl_t == 0);
            int nfit = 0;
            unsigned allv = 0u;
            const int ntr = produce_stage<false, 0>(
                sm.buf[slot], sm.meta[slot], &sm.full[slot], P.traces, P.trace_off, P.h,
                nullptr, P.list, lbeg, M, pl_t, dt, 0.f, n_first, n_last,
                StageBounds{0.f, 0.f, 0.f, 0.f, bC0, bC1}, P.status, nfit, allv);
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
    const int n = lane_row0 + lane;
    const bool act = n >= 0 && n < nrows;
    const bool out = act && lane >= HW && lane < HW + kT;
    const RowConst rc = row_const(act, n);
    TwAccum a;
    #pragma unroll
    for (int r = 0; r < kTwR; ++r) a.cidx[r] = INT_MAX;
    float bestS = -1.f, bestT = 0.f;
    int bestC = INT_MAX;
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
                a.cidx[r] = c;
                a.Cr[r] = c < P.ncand ? P.C[c] : 0.f;
                a.s[r] = 0.f;
                a.e[r] = 0.f;
                a.M[r] = 0;
            }
        }
        const int ntr = min(d.ntr, kChunkT);
        const int slot_base = (int)(reinterpret_cast<const float*>(sm.buf[slot]) - smf);
        if (ntr > 0 && a.cidx[0] < P.ncand) {
            int t = 0;
            while (t < ntr) {                          // runs of check-free / checked traces
                const bool fast = (d.allv >> t) & 1u;
                const unsigned rest = (fast ? ~d.allv : d.allv) >> t;
                const int len = rest ? __ffs(rest) - 1 : 32;
                const int t1 = min(ntr, t + len);
                if (fast) tw_run<true>(a, sm.meta[slot], t, t1, slot_base, rc, zidx, smf);
                else tw_run<false>(a, sm.meta[slot], t, t1, slot_base, rc, zidx, smf);
                t = t1;
            }
        }
        if (d.last) {
            #pragma unroll
            for (int r = 0; r < kTwR; ++r) {
                const int c = a.cidx[r];
                // inactive rows contributed nothing, so their s, e, M are 0
                const float sr = act ? a.s[r] : 0.f;
                const float me = act ? (float)a.M[r] * a.e[r] : 0.f;
                float num, den;
                window_sums<HW>(sr, me, lane, num, den);
                if (c >= P.ncand || !out) continue;
                const float sv = den > 0.f ? num / den : 0.f;
                const float st = a.M[r] > 0 ? a.s[r] / (float)a.M[r] : 0.f;
                if (P.S_cube) P.S_cube[(row0 + n) * (int64_t)P.ncand + c] = sv;
                if (sv > bestS) { bestS = sv; bestC = c; bestT = st; }
            }
        }
        mbar_arrive(&sm.empty[slot]);
    }

    sm.redS[warp][lane] = bestS;
    sm.redC[warp][lane] = bestC;
    sm.redT[warp][lane] = bestT;
    consumer_bar(32 * kTwWarps);
    if (aborted || sm.abort_flag) return;
    if (warp == 0 && out) {
        float bs, bt;
        int bc;
        reduce_best(sm, kTwWarps, lane, bs, bc, bt);
        const int64_t row = row0 + n;
        P.best_idx[row] = bc;
        P.best_S[row] = bs;
        P.stack[row] = bt;
        if (P.best_param) P.best_param[row] = P.C[bc];
    }
}

template <int W>
cudaError_t launch_t0win_w(SearchParams p, int max_rows, cudaStream_t stream) {
    static bool configured[64] = {};
    const int smem = (int)sizeof(SearchSmem);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(t0win_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    constexpr int kT = 32 - 2 * (W / 2);
    p.tiles_per_owner = (max_rows + kT - 1) / kT;
    const int64_t grid = p.nowner * (int64_t)p.tiles_per_owner;
    if (grid <= 0) return cudaSuccess;
    if (grid > INT_MAX) return cudaErrorInvalidValue;
    t0win_kernel<W><<<(unsigned)grid, kTwThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_t0win(const SearchParams& p, int w, int max_rows, cudaStream_t s) {
    switch (w) {
        case 1: return launch_t0win_w<1>(p, max_rows, s);
        case 3: return launch_t0win_w<3>(p, max_rows, s);
        case 5: return launch_t0win_w<5>(p, max_rows, s);
        case 7: return launch_t0win_w<7>(p, max_rows, s);
        case 9: return launch_t0win_w<9>(p, max_rows, s);
        case 11: return launch_t0win_w<11>(p, max_rows, s);
        case 13: return launch_t0win_w<13>(p, max_rows, s);
        case 15: return launch_t0win_w<15>(p, max_rows, s);
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
    cudaError_t e = launch_t0win(p, w, d->max_rows, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cmp_semblance_t0win launch");
    return SEIS_OK;
}
