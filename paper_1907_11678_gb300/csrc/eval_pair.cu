// eval_pair.cu -- semblance, stack and the adjoint dS/d(A,B,C) of TWO CRS operators per
// output row in one pass (the evaluations of a multi-start refinement, two starts at a time).
//
// It computes exactly what eval_kernel<CRS, W, GRAD> computes for each of the two operators
// (Eq. 1 and Algorithm 1 at the operator; the chain rule through the CRS traveltime of
// Section 2.2 and the linear interpolation, k and the participation mask held fixed), with
// the same operations in the same order, so every output is bit-identical to two separate
// evaluations.  The two operators of a row occupy the two halves of Blackwell's packed
// f32x2 instructions: one issue slot serves both, and every staged trace window serves
// 2 x 128 (row, operator) pairs instead of 128.
#include "search_kernel.cuh"
#include "eval_pair.h"

namespace seis {

constexpr int kPairWarps = 4;
constexpr int kPairThreads = 32 * (kPairWarps + 1);
constexpr int kPairConsumers = 32 * kPairWarps;
constexpr int kPairRows = 32 * kPairWarps;       // rows per CTA, as the single kernel
constexpr int kPairSlots = 2;
constexpr int kPairCTAs = 3;                     // register-limited (two operators' sums)

struct PairSmem {
    float buf[kPairSlots][kBuf];
    TraceMeta meta[kPairSlots][kChunkT];
    StageDesc desc[kPairSlots];
    uint64_t full[kPairSlots];
    uint64_t empty[kPairSlots];
    float zeros[16];
    int abort_flag;
    int pad[3];
};

template <int W>
__global__ void __launch_bounds__(kPairThreads, kPairCTAs) eval_pair_kernel(const EvalPairParams Q) {
    constexpr int HW = W / 2;
    const EvalParams& P = Q.p;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PairSmem& sm = *reinterpret_cast<PairSmem*>(smem_raw);
    const float* smf = reinterpret_cast<const float*>(smem_raw);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t owner = blockIdx.x / P.tiles_per_owner;
    const int tile = (int)(blockIdx.x - owner * P.tiles_per_owner);
    if (owner >= P.nowner) return;
    const int64_t row0 = P.out_off[owner];
    const int nrows = (int)(P.out_off[owner + 1] - row0);
    const int n0 = tile * kPairRows;
    if (n0 >= nrows) return;
    const int64_t lbeg = P.list_off[owner];
    const int64_t M64 = P.list_off[owner + 1] - lbeg;
    const int M = M64 < 0 ? 0 : (M64 > INT_MAX ? INT_MAX : (int)M64);
    const float dt = P.dt[owner];

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPairSlots; ++s) {
            mbar_init(&sm.full[s], 32);
            mbar_init(&sm.empty[s], kPairConsumers);
        }
        sm.abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 16) sm.zeros[threadIdx.x] = 0.f;
    __syncthreads();

    if (warp == kPairWarps) {
        // ---------------- producer: windows for the union of both operator sets ----------
        const float mc = P.m_c[owner];
        const int n_last = min(n0 + kPairRows - 1, nrows - 1);
        float lA0 = FLT_MAX, lA1 = -FLT_MAX, lB0 = FLT_MAX, lB1 = -FLT_MAX, lC0 = FLT_MAX,
              lC1 = -FLT_MAX;
        for (int n = n0 + lane; n <= n_last; n += 32) {
            for (int k = 0; k < 2; ++k) {
                const float* th = (k ? Q.theta2 : P.theta) + (row0 + n) * 3;
                lA0 = fminf(lA0, th[0]); lA1 = fmaxf(lA1, th[0]);
                lB0 = fminf(lB0, th[1]); lB1 = fmaxf(lB1, th[1]);
                lC0 = fminf(lC0, th[2]); lC1 = fmaxf(lC1, th[2]);
            }
        }
        const StageBounds bnd{warp_min(lA0), warp_max(lA1), warp_min(lB0), warp_max(lB1),
                              warp_min(lC0), warp_max(lC1)};
        int pl_t = 0;
        bool done = false;
        int s = 0;
        for (;; ++s) {
            const int slot = s % kPairSlots;
            if (s >= kPairSlots && !sm.abort_flag) {
                if (!mbar_wait_backoff(&sm.empty[slot], (uint32_t)(((s / kPairSlots) & 1) ^ 1))) {
                    sm.abort_flag = 1;
                    record_status(P.status, kStatusTimeout);
                }
            }
            __syncwarp();
            if (sm.abort_flag || done) {
                if (lane == 0) sm.desc[slot] = make_desc(0, 0, 0u, 0, 0, 1);
                __syncwarp();
                mbar_arrive(&sm.full[slot]);
                break;
            }
            int nfit = 0;
            unsigned allv = 0u;
            const int ntr = produce_stage<true, HW>(sm.buf[slot], (int)(sm.buf[slot] - smf),
                                                    sm.meta[slot], &sm.full[slot], P.traces,
                                                    P.trace_off, P.h, P.m, P.list, lbeg,
                                                    M, pl_t, dt, mc, n0, n_last, bnd, P.status,
                                                    nfit, allv);
            pl_t += nfit;
            done = pl_t >= M;
            if (lane == 0) sm.desc[slot] = make_desc(0, ntr, allv, 0, 0, 0);
            __syncwarp();
            mbar_arrive(&sm.full[slot]);
        }
        const int s_end = s;
        for (int s2 = max(0, s_end - kPairSlots + 1); s2 <= s_end; ++s2)
            mbar_wait_bounded(&sm.full[s2 % kPairSlots], (uint32_t)((s2 / kPairSlots) & 1));
        return;
    }

    // ---------------- consumers: lane = row, operators (a, b) in the two f32x2 halves -----
    const int zidx = (int)(reinterpret_cast<const float*>(sm.zeros) - smf);
    const int nrow = n0 + warp * 32 + lane;
    const bool act = nrow < nrows;
    const int n = act ? nrow : (1 << 24);
    const float nf = fmaxf((float)n, 1e-30f);
    const f2_t nf2 = pk2(nf, nf);
    float Aa = 0.f, Ba = 0.f, Ca = 0.f, Ab = 0.f, Bb = 0.f, Cb = 0.f;
    if (act) {
        const float* ta = P.theta + (row0 + nrow) * 3;
        const float* tb = Q.theta2 + (row0 + nrow) * 3;
        Aa = ta[0]; Ba = ta[1]; Ca = ta[2];
        Ab = tb[0]; Bb = tb[1]; Cb = tb[2];
    }
    const f2_t A2 = pk2(Aa, Ab), B2 = pk2(Ba, Bb), C2 = pk2(Ca, Cb);
    f2_t num[W], dnum[3][W];
    f2_t den = 0ull;
    f2_t dden[3] = {0ull, 0ull, 0ull};
    int cnta = 0, cntb = 0;
    #pragma unroll
    for (int j = 0; j < W; ++j) {
        num[j] = 0ull;
        #pragma unroll
        for (int a = 0; a < 3; ++a) dnum[a][j] = 0ull;
    }
    bool aborted = false;
    const f2_t shift2 = pk2(kFloorShift, kFloorShift);

    for (int s = 0;; ++s) {
        const int slot = s % kPairSlots;
        if (!mbar_wait_bounded(&sm.full[slot], (uint32_t)((s / kPairSlots) & 1))) {
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
        const int ntr = min(d.ntr, kChunkT);
        // One staged trace.  FAST: the producer found that every row and operator of the CTA
        // takes part (window inside the trace, t0 + A dm >= 1e-3 and t^2 >= 1 sample^2 over
        // the operators' box), so the participation tests, the selects and the guard on
        // sqrt(t^2) + p are left out; the results are those of the checked form.
        auto trace = [&](int t, auto fast) {
            constexpr bool FAST = decltype(fast)::value;
            const TraceConst tc = trace_const(sm.meta[slot][t], n);
            // traveltime of both operators (the single kernel's operations, lane-wise)
            const f2_t e2 = tc.e2;
            const f2_t a2 = mul2(A2, e2);
            const f2_t pp2 = add2(nf2, a2);
            const f2_t rr2 = fma2(B2, tc.g2, mul2(C2, tc.q2));
            const f2_t rad2 = fma2(pp2, pp2, rr2);
            float ra, rb, pa, pb;
            up2(rad2, ra, rb);
            up2(pp2, pa, pb);
            const float sua = sqrt_fast(ra), sub = sqrt_fast(rb);
            float sa, sb;
            up2(add2(pk2(sua, sub), pp2), sa, sb);
            if constexpr (!FAST) {
                sa = fmaxf(sa, 1e-30f);
                sb = fmaxf(sb, 1e-30f);
            }
            const f2_t D2 = fma2(rr2, pk2(rcp_fast(sa), rcp_fast(sb)), a2);
            const f2_t t2 = add2_rm(D2, shift2);
            float ta, tb;
            up2(t2, ta, tb);
            f2_t x2 = sub2(D2, sub2(t2, shift2));
            const int kka = __float_as_int(ta) + tc.off;
            const int kkb = __float_as_int(tb) + tc.off;
            int ia, ib;
            f2_t ru2;
            if constexpr (FAST) {
                // kk is clamped only to keep the reads of rows past the owner's end inside
                // the staged window (their sums are discarded)
                ia = tc.kbase + (int)min((unsigned)kka, tc.rng);
                ib = tc.kbase + (int)min((unsigned)kkb, tc.rng);
                ru2 = pk2(rcp_fast(sua), rcp_fast(sub));
            } else {
                const bool oka = pa >= 0.f && (unsigned)kka <= tc.rng;
                const bool okb = pb >= 0.f && (unsigned)kkb <= tc.rng;
                float xa, xb;
                up2(x2, xa, xb);
                x2 = pk2(oka ? xa : 0.f, okb ? xb : 0.f);
                ia = oka ? tc.kbase + kka : zidx;
                ib = okb ? tc.kbase + kkb : zidx;
                cnta += oka ? 1 : 0;
                cntb += okb ? 1 : 0;
                ru2 = pk2((oka && sua > 0.f) ? rcp_fast(sua) : 0.f,
                          (okb && sub > 0.f) ? rcp_fast(sub) : 0.f);
            }
            // du/d(A, B, C) of both operators, B's and C's taken at twice the single kernel's
            // (g ru and q ru instead of 0.5 g ru and 0.5 q ru): that is the factor 2 their
            // energy terms need, and their numerator sums come out doubled, which the end
            // accounts for exactly (v (2 dnum) = (2 v) dnum).  A's energy term is summed
            // without its factor 2 and doubled once after the loop (x + x, exact).  Powers of
            // two only, so every output is still bit-identical to the single kernel's.
            f2_t du[3];
            du[0] = mul2(mul2(pp2, e2), ru2);
            du[1] = mul2(tc.g2, ru2);
            du[2] = mul2(tc.q2, ru2);
            float FA[W + 1], FB[W + 1];
            #pragma unroll
            for (int j = 0; j <= W; ++j) { FA[j] = smf[ia + j]; FB[j] = smf[ib + j]; }
            f2_t vd = 0ull;
            #pragma unroll
            for (int j = 0; j < W; ++j) {
                const f2_t f0 = pk2(FA[j], FB[j]);
                const f2_t dj = sub2(pk2(FA[j + 1], FB[j + 1]), f0);
                const f2_t v = fma2(x2, dj, f0);
                num[j] = add2(num[j], v);
                den = fma2(v, v, den);
                vd = fma2(v, dj, vd);
                #pragma unroll
                for (int a = 0; a < 3; ++a) dnum[a][j] = fma2(dj, du[a], dnum[a][j]);
            }
            #pragma unroll
            for (int a = 0; a < 3; ++a) dden[a] = fma2(du[a], vd, dden[a]);
        };
        int t = 0;
        while (t < ntr) {                      // runs of check-free / checked traces
            const bool fast = (d.allv >> t) & 1u;
            const unsigned rest = (fast ? ~d.allv : d.allv) >> t;
            const int len = rest ? __ffs(rest) - 1 : 32;
            const int t1 = min(ntr, t + len);
            if (fast) {
                for (int u = t; u < t1; ++u) trace(u, std::true_type{});
                cnta += t1 - t;
                cntb += t1 - t;
            } else {
                for (int u = t; u < t1; ++u) trace(u, std::false_type{});
            }
            t = t1;
        }
        mbar_arrive(&sm.empty[slot]);
    }
    if (aborted || !act) return;
    dden[0] = add2(dden[0], dden[0]);                // A's energy term: the factor 2

    // Eq. 1, the stack and dS per operator, in the single kernel's order
    #pragma unroll
    for (int k = 0; k < 2; ++k) {
        float nu = 0.f, ac = 0.f;
        float dnu[3] = {0.f, 0.f, 0.f};
        #pragma unroll
        for (int j = 0; j < W; ++j) {
            float lo, hi;
            up2(num[j], lo, hi);
            const float v = k ? hi : lo;
            nu = fmaf(v, v, nu);
            ac += v;
            // B's and C's dnum hold twice the single kernel's sums: 2 v dnum = v (2 dnum)
            up2(dnum[0][j], lo, hi);
            dnu[0] = fmaf(2.f * v, k ? hi : lo, dnu[0]);
            #pragma unroll
            for (int a = 1; a < 3; ++a) {
                up2(dnum[a][j], lo, hi);
                dnu[a] = fmaf(v, k ? hi : lo, dnu[a]);
            }
        }
        float dl, dh;
        up2(den, dl, dh);
        const float dn = (k ? dh : dl) + 0.f;
        const int cnt = k ? cntb : cnta;
        const float Nf = (float)cnt;
        const bool live = cnt > 0 && dn > 0.f;
        const float Sv = live ? nu / (Nf * dn) : 0.f;
        const int64_t row = row0 + nrow;
        float* Sout = k ? Q.S2 : P.S;
        float* Stk = k ? Q.stack2 : P.stack;
        float* G = k ? Q.grad2 : P.grad;
        if (Sout) Sout[row] = Sv;
        if (Stk) Stk[row] = cnt > 0 ? ac / (Nf * (float)W) : 0.f;
        if (G) {
            #pragma unroll
            for (int a = 0; a < 3; ++a) {
                float gl, gh;
                up2(dden[a], gl, gh);
                G[row * 3 + a] = live ? (dnu[a] - Sv * Nf * (k ? gh : gl)) / (Nf * dn) : 0.f;
            }
        }
    }
}

template <int W>
static cudaError_t launch_pair_w(const EvalPairParams& q, cudaStream_t stream) {
    static bool configured[64] = {};
    const int smem = (int)sizeof(PairSmem);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(eval_pair_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    const int64_t grid = q.p.nowner * (int64_t)q.p.tiles_per_owner;
    if (grid <= 0) return cudaSuccess;
    if (grid > INT_MAX) return cudaErrorInvalidValue;
    eval_pair_kernel<W><<<(unsigned)grid, kPairThreads, smem, stream>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_eval_pair(const EvalPairParams& q, int w, cudaStream_t s) {
    switch (w) {
        case 1: return launch_pair_w<1>(q, s);
        case 3: return launch_pair_w<3>(q, s);
        case 5: return launch_pair_w<5>(q, s);
        case 7: return launch_pair_w<7>(q, s);
        case 9: return launch_pair_w<9>(q, s);
        case 11: return launch_pair_w<11>(q, s);
        case 13: return launch_pair_w<13>(q, s);
        case 15: return launch_pair_w<15>(q, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace seis
