// eval_kernel.cu -- semblance, stack and the analytic adjoint dS/d(A,B,C) of ONE operator per
// output row (the `stack`, `crs_semblance_grad` and `crs_refine` entry points), plus the
// update step of the gradient-ascent refinement.
//
// What it computes: Eq. 1 and Algorithm 1 (arXiv:1907.11678) at a given operator per row;
// the stack is Algorithm 1's linear accumulator at that operator.  The adjoint is the chain
// rule through the traveltime u(A,B,C) (CRS surface of Section 2.2, in samples:
// u^2 = (n + A dm/dt)^2 + B dm^2/dt^2 + C h^2/dt^2) and the linear interpolation, with k and
// the participation mask held fixed (derivative almost everywhere):
//   du/dA = p e / u, du/dB = g / (2u), du/dC = q / (2u)   (p = n + A e, e = dm/dt, g = e^2,
//                                                           q = h^2/dt^2)
//   dv_j = (f[k+j+1] - f[k+j]) du,  dnum_j = sum_i dv_ij,  dden = 2 sum_ij v_ij dv_ij,
//   dS = (2 sum_j num_j dnum_j - S N dden) / (N den).
// Layout: one CTA = one owner x 128 consecutive rows (4 consumer warps, lane = row) plus
// the producer warp of the search kernel, which stages each trace's window for the union of
// the CTA's operators through a two-slot bulk-copy ring (so that four CTAs share an SM).
#include "search_kernel.cuh"

namespace seis {

constexpr int kEvalWarps = 4;
constexpr int kEvalThreads = 32 * (kEvalWarps + 1);
constexpr int kEvalConsumers = 32 * kEvalWarps;
constexpr int kEvalRows = 32 * kEvalWarps;
constexpr int kEvalSlots = 2;           // ring depth: four CTAs (20 warps) fit an SM
constexpr int kEvalCTAs = 4;

// Shared memory of one CTA: the search kernel's slot layout with a two-slot ring.
struct EvalSmem {
    float buf[kEvalSlots][kBuf];
    TraceMeta meta[kEvalSlots][kChunkT];
    StageDesc desc[kEvalSlots];
    uint64_t full[kEvalSlots];
    uint64_t empty[kEvalSlots];
    float zeros[16];
    int abort_flag;
    int pad[3];
};

template <bool CRS, int W, bool GRAD>
__global__ void __launch_bounds__(kEvalThreads, kEvalCTAs) eval_kernel(const EvalParams P) {
    constexpr int HW = W / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    EvalSmem& sm = *reinterpret_cast<EvalSmem*>(smem_raw);
    const float* smf = reinterpret_cast<const float*>(smem_raw);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t owner = blockIdx.x / P.tiles_per_owner;
    const int tile = (int)(blockIdx.x - owner * P.tiles_per_owner);
    if (owner >= P.nowner) return;
    const int64_t row0 = P.out_off[owner];
    const int nrows = (int)(P.out_off[owner + 1] - row0);
    const int n0 = tile * kEvalRows;
    if (n0 >= nrows) return;
    const int64_t lbeg = P.list_off[owner];
    const int64_t M64 = P.list_off[owner + 1] - lbeg;
    const int M = M64 < 0 ? 0 : (M64 > INT_MAX ? INT_MAX : (int)M64);
    const float dt = P.dt[owner];

    if (threadIdx.x == 0) {
        for (int s = 0; s < kEvalSlots; ++s) {
            mbar_init(&sm.full[s], 32);
            mbar_init(&sm.empty[s], kEvalConsumers);
        }
        sm.abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 16) sm.zeros[threadIdx.x] = 0.f;
    __syncthreads();

    auto theta_of = [&](int n, float& a, float& b, float& c) {
        const float* th = P.theta + (row0 + n) * (int64_t)P.nparam;
        if (P.nparam == 3) { a = th[0]; b = th[1]; c = th[2]; }
        else { a = 0.f; b = 0.f; c = th[0]; }
    };

    if (warp == kEvalWarps) {
        // ---------------- producer: one pass over the traces ----------------------------
        const float mc = CRS ? P.m_c[owner] : 0.f;
        const int n_last = min(n0 + kEvalRows - 1, nrows - 1);
        float lA0 = FLT_MAX, lA1 = -FLT_MAX, lB0 = FLT_MAX, lB1 = -FLT_MAX, lC0 = FLT_MAX,
              lC1 = -FLT_MAX;
        for (int n = n0 + lane; n <= n_last; n += 32) {
            float a, b, c;
            theta_of(n, a, b, c);
            lA0 = fminf(lA0, a); lA1 = fmaxf(lA1, a);
            lB0 = fminf(lB0, b); lB1 = fmaxf(lB1, b);
            lC0 = fminf(lC0, c); lC1 = fmaxf(lC1, c);
        }
        const StageBounds bnd{warp_min(lA0), warp_max(lA1), warp_min(lB0), warp_max(lB1),
                              warp_min(lC0), warp_max(lC1)};
        int pl_t = 0;
        bool done = false;
        int s = 0;
        for (;; ++s) {
            const int slot = s % kEvalSlots;
            if (s >= kEvalSlots && !sm.abort_flag) {
                if (!mbar_wait_backoff(&sm.empty[slot], (uint32_t)(((s / kEvalSlots) & 1) ^ 1))) {
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
            unsigned allv = 0u;                 // unused: this kernel checks every pair
            const int ntr = produce_stage<CRS, HW>(sm.buf[slot], (int)(sm.buf[slot] - smf),
                                                   sm.meta[slot], &sm.full[slot], P.traces,
                                                   P.trace_off, P.h, P.m, P.list, lbeg,
                                                   M, pl_t, dt, mc, n0, n_last, bnd, P.status,
                                                   nfit, allv);
            pl_t += nfit;
            done = pl_t >= M;
            if (lane == 0) sm.desc[slot] = make_desc(0, ntr, 0u, 0, 0, 0);
            __syncwarp();
            mbar_arrive(&sm.full[slot]);
        }
        const int s_end = s;
        for (int s2 = max(0, s_end - kEvalSlots + 1); s2 <= s_end; ++s2)
            mbar_wait_bounded(&sm.full[s2 % kEvalSlots], (uint32_t)((s2 / kEvalSlots) & 1));
        return;
    }

    // ---------------- consumers: lane = row, one operator each --------------------------
    const int zidx = (int)(reinterpret_cast<const float*>(sm.zeros) - smf);
    const int nrow = n0 + warp * 32 + lane;
    const bool act = nrow < nrows;
    const int n = act ? nrow : (1 << 24);
    const float nf = fmaxf((float)n, 1e-30f);
    const float nsq = nf * nf;
    float A = 0.f, B = 0.f, C = 0.f;
    if (act) theta_of(nrow, A, B, C);
    float num[W], dnum[GRAD ? 3 : 1][W];
    float den[2] = {0.f, 0.f};
    float dden[3] = {0.f, 0.f, 0.f};
    int cnt = 0;
    #pragma unroll
    for (int j = 0; j < W; ++j) {
        num[j] = 0.f;
        #pragma unroll
        for (int a = 0; a < (GRAD ? 3 : 1); ++a) dnum[a][j] = 0.f;
    }
    bool aborted = false;

    for (int s = 0;; ++s) {
        const int slot = s % kEvalSlots;
        if (!mbar_wait_bounded(&sm.full[slot], (uint32_t)((s / kEvalSlots) & 1))) {
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
        for (int t = 0; t < ntr; ++t) {
            const TraceConst tc = trace_const(sm.meta[slot][t], n);
            // traveltime (as the search kernel) plus, for the adjoint, du/d(A,B,C)
            float D, s_u, pp = nf;
            bool p_ok = true;
            if (CRS) {
                const float a = A * tc.e;
                pp = nf + a;
                const float rr = fmaf(B, tc.g, C * tc.q);
                const float rad = fmaf(pp, pp, rr);
                p_ok = pp >= 0.f;
                s_u = sqrt_fast(rad);
                D = fmaf(rr, rcp_fast(fmaxf(s_u + pp, 1e-30f)), a);
            } else {
                const float cq = C * tc.q;
                s_u = sqrt_fast(nsq + cq);
                D = cq * rcp_fast(s_u + nf);
            }
            const float tt = __fadd_rd(D, kFloorShift);
            const int kk = __float_as_int(tt) + tc.off;
            const bool ok = p_ok && (unsigned)kk <= tc.rng;
            const float x = ok ? D - (tt - kFloorShift) : 0.f;
            const int idx = ok ? tc.kbase + kk : zidx;
            cnt += ok ? 1 : 0;
            float du[3] = {0.f, 0.f, 0.f};
            if (GRAD) {
                const float ru = (ok && s_u > 0.f) ? rcp_fast(s_u) : 0.f;
                du[0] = pp * tc.e * ru;
                du[1] = 0.5f * tc.g * ru;
                du[2] = 0.5f * tc.q * ru;
            }
            float F[W + 1];
            #pragma unroll
            for (int j = 0; j <= W; ++j) F[j] = smf[idx + j];
            float vd = 0.f;
            #pragma unroll
            for (int j = 0; j < W; ++j) {
                const float dj = F[j + 1] - F[j];
                const float v = fmaf(x, dj, F[j]);
                num[j] += v;
                den[kDenChains == 2 ? (j & 1) : 0] = fmaf(v, v, den[kDenChains == 2 ? (j & 1) : 0]);
                if (GRAD) {
                    vd = fmaf(v, dj, vd);
                    #pragma unroll
                    for (int a = 0; a < 3; ++a) dnum[a][j] = fmaf(dj, du[a], dnum[a][j]);
                }
            }
            if (GRAD) {
                #pragma unroll
                for (int a = 0; a < 3; ++a) dden[a] = fmaf(2.f * du[a], vd, dden[a]);
            }
        }
        mbar_arrive(&sm.empty[slot]);
    }
    if (aborted || !act) return;

    float nu0 = 0.f, nu1 = 0.f, ac = 0.f;
    float dnu[3] = {0.f, 0.f, 0.f};
    #pragma unroll
    for (int j = 0; j < W; ++j) {
        if (kDenChains == 2 && (j & 1)) nu1 = fmaf(num[j], num[j], nu1);
        else nu0 = fmaf(num[j], num[j], nu0);
        ac += num[j];
        if (GRAD) {
            #pragma unroll
            for (int a = 0; a < 3; ++a) dnu[a] = fmaf(2.f * num[j], dnum[a][j], dnu[a]);
        }
    }
    const float nu = nu0 + nu1, dn = den[0] + den[1];
    const float Nf = (float)cnt;
    const bool live = cnt > 0 && dn > 0.f;
    const float Sv = live ? nu / (Nf * dn) : 0.f;
    const int64_t row = row0 + nrow;
    if (P.S) P.S[row] = Sv;
    if (P.stack) P.stack[row] = cnt > 0 ? ac / (Nf * (float)W) : 0.f;
    if (P.N) P.N[row] = cnt;
    if (GRAD && P.grad) {
        #pragma unroll
        for (int a = 0; a < 3; ++a)
            P.grad[row * 3 + a] = live ? (dnu[a] - Sv * Nf * dden[a]) / (Nf * dn) : 0.f;
    }
}

// Inverse curvature estimate of one row, symmetric 3x3 stored as H00 H01 H02 H11 H12 H22.
__device__ __forceinline__ void h_reset(float* H, const float* gz, float step0) {
    const float gn = sqrtf(gz[0] * gz[0] + gz[1] * gz[1] + gz[2] * gz[2]);
    const float h0 = gn > 0.f ? step0 / gn : 0.f;
    H[0] = h0; H[1] = 0.f; H[2] = 0.f; H[3] = h0; H[4] = 0.f; H[5] = h0;
}

__device__ __forceinline__ void h_mul(const float* H, const float* v, float* o) {
    o[0] = H[0] * v[0] + H[1] * v[1] + H[2] * v[2];
    o[1] = H[1] * v[0] + H[3] * v[1] + H[4] * v[2];
    o[2] = H[2] * v[0] + H[4] * v[1] + H[5] * v[2];
}

// One refinement step per row: assess the evaluated trial, then propose the next one.  The
// rule is a projected quasi-Newton (BFGS) ascent of S in normalised coordinates
// z = (theta - lo) / (hi - lo) with step halving on a failed trial:
//   d = H g (H reset to (step0/|g|) I when d is not an ascent direction), |d| <= 0.25,
//   trial z + a d clamped to [0, 1]; an accepted trial updates H with the expanded BFGS
//   inverse update  H += -rho (u s' + s u') + (rho + rho^2 y.u) s s',  u = H y,
//   rho = 1/(s.y), s = step, y = g - g' (gradient change of -S), when s.y > 1e-6 |s||y|,
//   and resets a to 1; a failed trial halves a.  step[] holds a (-1 once g vanished).
__global__ void refine_update_kernel(const RefineParams R) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= R.rows) return;
    float span[3], H[6];
    for (int a = 0; a < 3; ++a) span[a] = R.hi[a] - R.lo[a];
    float al = R.init ? 1.f : R.step[r];
    if (R.init) {
        float gz[3];
        R.S[r] = R.trial_S[r];
        R.stack[r] = R.trial_stack[r];
        for (int a = 0; a < 3; ++a) {
            R.grad[r * 3 + a] = R.trial_grad[r * 3 + a];
            gz[a] = R.trial_grad[r * 3 + a] * span[a];
        }
        h_reset(H, gz, R.step0);
    } else {
        for (int i = 0; i < 6; ++i) H[i] = R.H[r * 6 + i];
        if (R.assess && al > 0.f) {
            if (R.trial_S[r] >= R.S[r]) {
                float sv[3], yv[3], ss = 0.f, yy = 0.f, sy = 0.f;
                for (int a = 0; a < 3; ++a) {
                    sv[a] = (R.trial_theta[r * 3 + a] - R.lo[a]) / span[a] -
                            (R.theta[r * 3 + a] - R.lo[a]) / span[a];
                    yv[a] = R.grad[r * 3 + a] * span[a] - R.trial_grad[r * 3 + a] * span[a];
                    ss = fmaf(sv[a], sv[a], ss);
                    yy = fmaf(yv[a], yv[a], yy);
                    sy = fmaf(sv[a], yv[a], sy);
                }
                if (sy > 1e-6f * sqrtf(ss) * sqrtf(yy)) {
                    float u[3];
                    h_mul(H, yv, u);
                    const float rho = 1.f / sy;
                    const float yu = yv[0] * u[0] + yv[1] * u[1] + yv[2] * u[2];
                    const float c = rho + rho * rho * yu;
                    const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
                    for (int k = 0; k < 6; ++k) {
                        const int i = ii[k], j = jj[k];
                        H[k] += -rho * (u[i] * sv[j] + sv[i] * u[j]) + c * sv[i] * sv[j];
                    }
                }
                R.S[r] = R.trial_S[r];
                R.stack[r] = R.trial_stack[r];
                for (int a = 0; a < 3; ++a) {
                    R.theta[r * 3 + a] = R.trial_theta[r * 3 + a];
                    R.grad[r * 3 + a] = R.trial_grad[r * 3 + a];
                }
                al = 1.f;
            } else {
                al *= 0.5f;
            }
        }
    }
    if (R.propose) {
        float gz[3], d[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < 3; ++a) gz[a] = R.grad[r * 3 + a] * span[a];
        const float gn = sqrtf(gz[0] * gz[0] + gz[1] * gz[1] + gz[2] * gz[2]);
        if (!(gn > 0.f)) al = -1.f;                  // stationary: stop
        if (al > 0.f) {
            h_mul(H, gz, d);
            if (!(d[0] * gz[0] + d[1] * gz[1] + d[2] * gz[2] > 0.f)) {
                h_reset(H, gz, R.step0);
                h_mul(H, gz, d);
            }
            const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (dn > 0.25f)
                for (int a = 0; a < 3; ++a) d[a] *= 0.25f / dn;
        }
        for (int a = 0; a < 3; ++a) {
            const float z = (R.theta[r * 3 + a] - R.lo[a]) / span[a];
            const float zt = fminf(fmaxf(z + al * d[a], 0.f), 1.f);
            R.trial_theta[r * 3 + a] = al > 0.f ? fmaf(zt, span[a], R.lo[a]) : R.theta[r * 3 + a];
        }
    }
    for (int i = 0; i < 6; ++i) R.H[r * 6 + i] = H[i];
    R.step[r] = al;
}

template <bool CRS, int W, bool GRAD>
static cudaError_t launch_eval_w(const EvalParams& p, cudaStream_t stream) {
    static bool configured[64] = {};
    const int smem = (int)sizeof(EvalSmem);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(eval_kernel<CRS, W, GRAD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    const int64_t grid = p.nowner * (int64_t)p.tiles_per_owner;
    if (grid <= 0) return cudaSuccess;
    if (grid > INT_MAX) return cudaErrorInvalidValue;
    eval_kernel<CRS, W, GRAD><<<(unsigned)grid, kEvalThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

template <bool CRS, bool GRAD>
static cudaError_t launch_eval_g(const EvalParams& p, int w, cudaStream_t s) {
    switch (w) {
        case 1: return launch_eval_w<CRS, 1, GRAD>(p, s);
        case 3: return launch_eval_w<CRS, 3, GRAD>(p, s);
        case 5: return launch_eval_w<CRS, 5, GRAD>(p, s);
        case 7: return launch_eval_w<CRS, 7, GRAD>(p, s);
        case 9: return launch_eval_w<CRS, 9, GRAD>(p, s);
        case 11: return launch_eval_w<CRS, 11, GRAD>(p, s);
        case 13: return launch_eval_w<CRS, 13, GRAD>(p, s);
        case 15: return launch_eval_w<CRS, 15, GRAD>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_eval(const EvalParams& p, bool crs, bool grad, int w, cudaStream_t s) {
    if (!crs) return grad ? cudaErrorInvalidValue : launch_eval_g<false, false>(p, w, s);
    return grad ? launch_eval_g<true, true>(p, w, s) : launch_eval_g<true, false>(p, w, s);
}

cudaError_t launch_refine_update(const RefineParams& r, cudaStream_t s) {
    if (r.rows <= 0) return cudaSuccess;
    const int64_t blocks = (r.rows + 255) / 256;
    if (blocks > INT_MAX) return cudaErrorInvalidValue;
    refine_update_kernel<<<(unsigned)blocks, 256, 0, s>>>(r);
    return cudaGetLastError();
}

int eval_tile_rows() { return kEvalRows; }

}  // namespace seis
