// search_kernel.cuh -- the semblance search kernel (CMP and CRS) for sm_103a.
//
// What it computes (arXiv:1907.11678): Section 2.1 / Eq. 1 (windowed semblance with the
// 1/N normalisation), Algorithm 1 (per (t0, candidate) pair: intersect every trace,
// interpolate v = (c[j+1]-c[j])*x + c[j] along the window, accumulate num[j], den and the
// linear stack), Section 3.2 (argmax over candidates, stack at the pick), and for CRS
// Section 2.2 / 3.5 (the aperture's traces and the A/B/C traveltime surface).
//
// How (GB300 design; it keeps the paper's Algorithm 2 idea -- one staged trace window
// reused by many (t0, candidate) pairs -- and realises it with the TMA engine):
//   - one CTA = one owner (CMP gather or CRS central CDP) x 32 consecutive output rows;
//     lane l of every consumer warp owns row n0 + l, so the 32 lanes of a warp read 32
//     nearby sample indices of the same trace (conflict-free, often broadcast);
//   - candidates are processed in passes of NWARP x R (SearchCfg; 30 for the 15-warp
//     shapes); a consumer thread keeps R candidates' accumulators (num[w], den, N) in
//     registers through the whole trace loop, in packed pairs updated with Blackwell's
//     fma/add.rn.f32x2 (two FP32 lanes per issue) or in scalar FP32;
//   - a dedicated producer warp streams, per pass, the traces through a 4-slot
//     shared-memory ring in stages of up to 32 traces: for every trace it computes the
//     exact sample window the stage's 32 rows x the pass's candidates can touch
//     (traveltime bounds at the box corners, +-2 samples of margin), copies it with one
//     1-D bulk copy (cp.async.bulk) plus at most 3+3 scalar edge loads, and writes the
//     trace's metadata in the form the consumers use (window index, k offset and range,
//     geometry factors as ready f32x2 pairs); "full" mbarriers count the bytes, "empty"
//     mbarriers return the slot; no block-wide barrier in the loop;
//   - the traveltime is formed in sample units as u = n + D with the cancellation-free
//     moveout D = C q / (sqrt(n^2 + C q) + n), q = (h/dt)^2 (CRS: D = a + r/(s + p)),
//     which keeps the interpolation fraction accurate to ~1e-4 samples in FP32;
//   - the inner loop is branch-free: a pair whose trace does not take part reads a
//     zero strip and adds nothing;
//   - the argmax over all candidates stays inside the CTA (each thread's running best in
//     its own entry of the shared reduction arrays, then a reduction over the consumer
//     warps), so no atomics and no cube.
#pragma once
#include <cfloat>
#include <climits>
#include <type_traits>
#include "seis_dev.cuh"
#include "seis_internal.h"

namespace seis {

constexpr int kMaxWarps = 15;                // consumer warps per CTA, at most
constexpr int kChunkT = 32;                  // traces per stage at most (one per producer lane)
constexpr int kSlots = 4;                    // ring depth
constexpr int kBuf = 6144;                   // floats per slot (24 KB)
constexpr unsigned kFull = 0xffffffffu;

// Arithmetic forms of the window accumulation.  Blackwell's packed f32x2 instructions
// issue once for two FP32 lanes but run only on the heavy FMA pipe; scalar FP32 runs on
// either FMA pipe but needs twice the issue slots.  The hybrids split each window
// sample's work between the two so that neither the issue slots nor the heavy pipe alone
// bound the kernel.
enum SearchMode : int {
    kScalar = 0,    // everything scalar
    kPacked = 1,    // traveltime and window in f32x2 pairs of candidates
    kHybridD = 2,   // scalar traveltime and sample difference; packed interpolation and sums
    kHybridV = 3,   // scalar traveltime, difference and interpolation; packed sums
};

// Tile shape and arithmetic form of one kernel variant (chosen by the autotuner):
// NWARP consumer warps + 1 producer warp per CTA, R candidates per consumer thread per
// pass, accumulation MODE.  Two CTAs per SM.
template <int NWARP, int R, int MODE>
struct SearchCfg {
    static constexpr int kWarps = NWARP;
    static constexpr int kR = R;
    static constexpr int kMode = MODE;
    static constexpr bool kPairs = MODE != kScalar;     // candidates processed in pairs
    static constexpr int kThreads = 32 * (NWARP + 1);
    static constexpr int kConsumers = 32 * NWARP;
    static constexpr int kCB = NWARP * R;     // candidates per pass
    static_assert(kCB <= 32, "the producer bounds one candidate per lane");
    static_assert(NWARP <= kMaxWarps, "reduction arrays are sized for kMaxWarps");
    static_assert(!kPairs || (R % 2) == 0, "candidate pairs need an even R");
};

// Per-trace metadata of one stage, written by the producer in the form the consumers use
// directly: the index arithmetic is folded into three integers, and the geometry factors
// are stored twice so that a packed f32x2 pair loads straight into a register pair.
struct __align__(16) TraceMeta {
    int kbase;      // shared-memory float index of the window of k = kmin (slot included)
    int offk;       // -(bits of the floor shift) - kmin: kk = bits(D + shift, rounded down)
                    //   + n + offk, and intersections with 0 <= kk <= rng take part (window
    unsigned rng;   //   inside the trace and inside the staged sample window); rng = kmax - kmin
    int pad0;
    float q, q_, e, e_;   // (h/dt)^2, dm/dt (CRS), each twice
    float g, g_;          // (dm/dt)^2 (CRS), twice
    int pad1, pad2;
};

struct __align__(16) StageDesc {
    int pass;          // candidate pass
    int ntr;           // traces staged (compacted, in list order)
    unsigned allv;     // bit t: every (row, candidate) of the stage takes part for trace t
    int first, last;   // first / last stage of the pass
    int end;           // no more stages
    int item, tile;    // batch kernel: the task
    int task_end;      // batch kernel: last stage of the task
    int ncand, nrows;  // batch kernel: candidates and output rows of the task's item
    int pad0;
};

__device__ __forceinline__ StageDesc make_desc(int pass, int ntr, unsigned allv, int first,
                                               int last, int end, int item = 0, int tile = 0,
                                               int task_end = 0, int ncand = 0, int nrows = 0) {
    return StageDesc{pass, ntr, allv, first, last, end, item, tile, task_end, ncand, nrows, 0};
}

struct SearchSmem {
    float buf[kSlots][kBuf];
    TraceMeta meta[kSlots][kChunkT];
    StageDesc desc[kSlots];
    uint64_t full[kSlots];
    uint64_t empty[kSlots];
    float zeros[16];
    int abort_flag;
    int pad[3];
    float redS[kMaxWarps][32];
    int redC[kMaxWarps][32];
    float redT[kMaxWarps][32];
};

// ---- packed FP32 pairs (Blackwell f32x2) -------------------------------------------
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t pk2(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(f2_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) {
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) {
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// a + b rounded toward -infinity (used for the floor below)
__device__ __forceinline__ f2_t add2_rm(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// floor() by rounding: for |D| < 2^22, D + 1.5*2^23 rounded toward -inf is
// 1.5*2^23 + floor(D) exactly, so its bit pattern minus that of 1.5*2^23 is floor(D) as an
// integer and subtracting 1.5*2^23 back gives floor(D) as a float.  Out-of-range or NaN D
// give huge positive or negative integers, which the range test rejects.
constexpr float kFloorShift = 12582912.0f;     // 1.5 * 2^23
constexpr int kFloorShiftBits = 0x4B400000;
// FMA chains of the window energy (and of the numerator's sum of squares, summed in the same
// order): 1 leaves the packed kernels two more registers (fewer spills in CRS) and costs the
// scalar ones some ILP; every kernel uses the same value, so all stay bit-identical.
constexpr int kDenChains = 1;

__device__ __forceinline__ float warp_min(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ void consumer_bar(int nthreads) {
    asm volatile("bar.sync 1, %0;" :: "r"(nthreads) : "memory");
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

// Per-trace constants of one consumer thread: with kk = k - kmin, the trace takes part iff
// 0 <= kk <= rng, and its window starts at shared-memory float index kbase + kk.  q2, e2
// and g2 hold each factor in both halves of a packed pair.
struct TraceConst {
    float q, e, g;
    f2_t q2, e2, g2;
    int off;        // n - kFloorShiftBits - kmin: kk = bits(D + shift, rounded down) + off
    unsigned rng;   // kmax - kmin
    int kbase;      // shared index of the window of k = kmin
};

__device__ __forceinline__ TraceConst trace_const(const TraceMeta& tm, int n) {
    TraceConst c;
    c.q = tm.q;
    c.e = tm.e;
    c.g = tm.g;
    c.q2 = *reinterpret_cast<const f2_t*>(&tm.q);
    c.e2 = *reinterpret_cast<const f2_t*>(&tm.e);
    c.g2 = *reinterpret_cast<const f2_t*>(&tm.g);
    c.off = n + tm.offk;
    c.rng = tm.rng;
    c.kbase = tm.kbase;
    return c;
}

// One intersection: traveltime -> (window start index, interpolation fraction, takes part).
// Rows past the owner's end carry n = 2^24 so that their k falls outside every trace.
template <bool CRS>
__device__ __forceinline__ void intersect_one(float A, float B, float C, const TraceConst& tc,
                                              float nf, float nsq, int zidx,
                                              int& idx, float& x, bool& ok) {
    float D;
    bool p_ok = true;
    if (CRS) {
        const float a = A * tc.e;
        const float pp = nf + a;
        const float rr = fmaf(B, tc.g, C * tc.q);
        const float rad = fmaf(pp, pp, rr);
        p_ok = pp >= 0.f;
        D = fmaf(rr, rcp_fast(fmaxf(sqrt_fast(rad) + pp, 1e-30f)), a);
    } else {
        const float cq = C * tc.q;
        D = cq * rcp_fast(sqrt_fast(nsq + cq) + nf);            // nf >= 1e-30
    }
    const float t = __fadd_rd(D, kFloorShift);
    const int kk = __float_as_int(t) + tc.off;
    ok = p_ok && (unsigned)kk <= tc.rng;
    x = ok ? D - (t - kFloorShift) : 0.f;
    idx = ok ? tc.kbase + kk : zidx;
}

// Two intersections (candidates a, b) with the traveltime arithmetic in f32x2 pairs.
template <bool CRS>
__device__ __forceinline__ void intersect_pair(f2_t A2, f2_t B2, f2_t C2, const TraceConst& tc,
                                               f2_t nf2, f2_t nsq2, int zidx,
                                               int& ia, int& ib, float& xa, float& xb,
                                               bool& oka, bool& okb) {
    const f2_t q2 = tc.q2;
    f2_t D2;
    bool pa_ok = true, pb_ok = true;
    if (CRS) {
        const f2_t a2 = mul2(A2, tc.e2);
        const f2_t pp2 = add2(nf2, a2);
        const f2_t rr2 = fma2(B2, tc.g2, mul2(C2, q2));
        const f2_t rad2 = fma2(pp2, pp2, rr2);
        float ra, rb, pa, pb;
        up2(rad2, ra, rb);
        up2(pp2, pa, pb);
        pa_ok = pa >= 0.f;
        pb_ok = pb >= 0.f;
        const f2_t sum2 = add2(pk2(sqrt_fast(ra), sqrt_fast(rb)), pp2);
        float sa, sb;
        up2(sum2, sa, sb);
        D2 = fma2(rr2, pk2(rcp_fast(fmaxf(sa, 1e-30f)), rcp_fast(fmaxf(sb, 1e-30f))), a2);
    } else {
        const f2_t cq2 = mul2(C2, q2);
        const f2_t rad2 = add2(nsq2, cq2);
        float ra, rb;
        up2(rad2, ra, rb);
        const f2_t sum2 = add2(pk2(sqrt_fast(ra), sqrt_fast(rb)), nf2);   // nf >= 1e-30
        float sa, sb;
        up2(sum2, sa, sb);
        D2 = mul2(cq2, pk2(rcp_fast(sa), rcp_fast(sb)));
    }
    const f2_t shift2 = pk2(kFloorShift, kFloorShift);
    const f2_t t2 = add2_rm(D2, shift2);
    const f2_t x2 = sub2(D2, sub2(t2, shift2));
    float ta, tb;
    up2(t2, ta, tb);
    up2(x2, xa, xb);
    const int kka = __float_as_int(ta) + tc.off;
    const int kkb = __float_as_int(tb) + tc.off;
    oka = pa_ok && (unsigned)kka <= tc.rng;
    okb = pb_ok && (unsigned)kkb <= tc.rng;
    xa = oka ? xa : 0.f;
    xb = okb ? xb : 0.f;
    ia = oka ? tc.kbase + kka : zidx;
    ib = okb ? tc.kbase + kkb : zidx;
}

// Window bounds of one stage: the extreme candidate parameters of the rows it serves.
struct StageBounds {
    float A0, A1, B0, B1, C0, C1;
};

// Producer warp, one stage: lane l takes trace pl_t + l of the owner's list, computes the
// sample window that rows n0..n_last x candidates within `b` can touch (traveltime bounds at
// the box corners, +-2 samples of margin), and the lanes whose windows fit the slot (a
// prefix) copy them: one cp.async.bulk of the 16-byte-aligned body plus scalar loads of at
// most 3 head and 3 tail samples.  Empty windows are left out; the metadata of the others is
// compacted into meta[0..ntr).  Returns ntr; nfit = traces consumed from the list.
template <bool CRS, int HW>
__device__ __forceinline__ int produce_stage(float* slotbuf, int slot_base, TraceMeta* meta,
                                             uint64_t* full,
                                             const float* traces, const int64_t* trace_off,
                                             const float* hh, const float* mm, const int32_t* list,
                                             int64_t lbeg, int M, int pl_t, float dt, float mc,
                                             int n0, int n_last, const StageBounds& b,
                                             unsigned* status, int& nfit_out,
                                             unsigned& allv_out) {
    const int lane = threadIdx.x & 31;
    const float bA0 = b.A0, bA1 = b.A1, bB0 = b.B0, bB1 = b.B1, bC0 = b.C0, bC1 = b.C1;
    fence_proxy_async_smem();   // earlier generic accesses of the slot before async writes
    const int t = pl_t + lane;
    const bool v = t < M;
    int len = 0, n_el = 0, mis = 0, lo = 0;
    bool allv = false;
    const float* src = nullptr;
    TraceMeta tm{};
    if (v) {
        const int64_t tid = list ? (int64_t)list[lbeg + t] : (lbeg + t);
        const int64_t toff = trace_off[tid];
        const int64_t ns64 = trace_off[tid + 1] - toff;
        const int ns_i = ns64 < 0 ? 0 : (ns64 > (INT_MAX / 4) ? (INT_MAX / 4) : (int)ns64);
        const double dtd = (double)dt;
        const double hd = (double)hh[tid];
        tm.q = (float)(hd * hd / (dtd * dtd));
        tm.q_ = tm.q;
        float aLo = 0.f, aHi = 0.f, rLo, rHi;
        if (CRS) {
            const double dm = mm ? (double)mm[tid] - (double)mc : 0.0;   // no midpoints: CMP
            tm.e = tm.e_ = (float)(dm / dtd);
            tm.g = tm.g_ = (float)(dm * dm / (dtd * dtd));
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
            const int klo = (int)floorf(uLo) - 2, khi = (int)floorf(uHi) + 2;
            const int kmin = max(klo, HW);
            const int kmax = min(khi, ns_i - HW - 2);
            // every pair of the box takes part: the traveltime is real with margin, and
            // the whole k range (with the +-2 margin) lies inside the trace's mask
            allv = klo >= HW && khi <= ns_i - HW - 2 && (!CRS || (float)n0 + aLo >= 1e-3f) &&
                   radLo >= 1.f;
            if (kmin <= kmax) {
                tm.offk = -kFloorShiftBits - kmin;
                tm.rng = (unsigned)(kmax - kmin);
                lo = kmin - HW;
                n_el = (kmax + HW + 1) - lo + 1;
                src = traces + toff + lo;
                mis = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
                len = (mis + n_el + 3) & ~3;
            }
        }
    }
    int pre = len;                                     // inclusive scan of lengths
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, pre, o);
        if (lane >= o) pre += y;
    }
    const bool fits = v && (pre <= kBuf);
    int nfit = __popc(__ballot_sync(kFull, fits));    // a prefix of the lanes
    // traces whose window is empty for this stage are left out of it
    const unsigned present = __ballot_sync(kFull, lane < nfit && n_el > 0);
    int ntr = __popc(present);
    const int pos = __popc(present & ((1u << lane) - 1u));
    allv_out = __reduce_or_sync(kFull, ((present >> lane) & 1u) && allv ? (1u << pos) : 0u);
    if (nfit == 0 && M > pl_t) {
        // a single window larger than a slot (traces are limited on the host so this
        // cannot happen): drop that trace and record it
        if (lane == 0) record_status(status, kStatusOverflow);
        nfit = 1;
        ntr = 0;
        allv_out = 0u;
    } else if (lane < nfit && n_el > 0) {
        const int off = pre - len;                       // multiple of 4 floats
        tm.kbase = slot_base + off + mis;      // the first staged sample, kmin - HW
        meta[pos] = tm;
        float* dst = slotbuf + off + mis;
        const int head = min((4 - mis) & 3, n_el);
        const int nb = (n_el - head) & ~3;
        if (nb > 0) {
            mbar_expect_tx(full, (uint32_t)nb * 4u);
            bulk_g2s(dst + head, src + head, (uint32_t)nb * 4u, full);
        }
        for (int e2 = 0; e2 < head; ++e2) dst[e2] = ldg_nc(src + e2);
        for (int e2 = head + nb; e2 < n_el; ++e2) dst[e2] = ldg_nc(src + e2);
    }
    nfit_out = nfit;
    return ntr;
}

// Check-free forms for traces on which every pair of the stage takes part: no mask test,
// no select, and for CRS no guard on sqrt(rad) + p, which the producer's test (rad >= 1,
// p >= 1e-3 over the stage's box) keeps at or above 1.  kk is clamped into the staged window only to keep every read inside it
// (rows past the owner's end and candidates past ncand land there; their sums are
// discarded).
template <bool CRS>
__device__ __forceinline__ void intersect_one_fast(float A, float B, float C, const TraceConst& tc,
                                                   float nf, float nsq, int& idx, float& x) {
    float D;
    if (CRS) {
        const float a = A * tc.e;
        const float pp = nf + a;
        const float rr = fmaf(B, tc.g, C * tc.q);
        D = fmaf(rr, rcp_fast(sqrt_fast(fmaf(pp, pp, rr)) + pp), a);   // >= 1: no guard
    } else {
        const float cq = C * tc.q;
        D = cq * rcp_fast(sqrt_fast(nsq + cq) + nf);
    }
    const float t = __fadd_rd(D, kFloorShift);
    const unsigned kk = min((unsigned)(__float_as_int(t) + tc.off), tc.rng);
    x = D - (t - kFloorShift);
    idx = tc.kbase + (int)kk;
}

template <bool CRS>
__device__ __forceinline__ void intersect_pair_fast(f2_t A2, f2_t B2, f2_t C2, const TraceConst& tc,
                                                    f2_t nf2, f2_t nsq2, int& ia, int& ib,
                                                    f2_t& x2) {
    const f2_t q2 = tc.q2;
    f2_t D2;
    if (CRS) {
        const f2_t a2 = mul2(A2, tc.e2);
        const f2_t pp2 = add2(nf2, a2);
        const f2_t rr2 = fma2(B2, tc.g2, mul2(C2, q2));
        const f2_t rad2 = fma2(pp2, pp2, rr2);
        float ra, rb;
        up2(rad2, ra, rb);
        const f2_t sum2 = add2(pk2(sqrt_fast(ra), sqrt_fast(rb)), pp2);
        float sa, sb;
        up2(sum2, sa, sb);
        D2 = fma2(rr2, pk2(rcp_fast(sa), rcp_fast(sb)), a2);      // sa, sb >= 1: no guard
    } else {
        const f2_t cq2 = mul2(C2, q2);
        const f2_t rad2 = add2(nsq2, cq2);
        float ra, rb;
        up2(rad2, ra, rb);
        const f2_t sum2 = add2(pk2(sqrt_fast(ra), sqrt_fast(rb)), nf2);
        float sa, sb;
        up2(sum2, sa, sb);
        D2 = mul2(cq2, pk2(rcp_fast(sa), rcp_fast(sb)));
    }
    const f2_t shift2 = pk2(kFloorShift, kFloorShift);
    const f2_t t2 = add2_rm(D2, shift2);
    x2 = sub2(D2, sub2(t2, shift2));                // fraction pair, kept packed
    float ta, tb;
    up2(t2, ta, tb);
    ia = tc.kbase + (int)min((unsigned)(__float_as_int(ta) + tc.off), tc.rng);
    ib = tc.kbase + (int)min((unsigned)(__float_as_int(tb) + tc.off), tc.rng);
}

// ---- consumer-side accumulation, shared by the search kernel and the batch kernel -----

// Per-thread accumulators of kR candidates for one output row.
template <int W, class CFG>
struct Accum {
    static constexpr bool kP = CFG::kPairs;
    static constexpr int kR = CFG::kR;
    static constexpr int kG = kP ? kR / 2 : kR;      // accumulator groups per thread
    f2_t num2[kP ? kG : 1][W];
    f2_t den2[kP ? kG : 1][2];                       // energy chains (kDenChains used)
    float num1[kP ? 1 : kG][W];
    float den1[kP ? 1 : kG][2];
    int cntv[kR];
    float Ar[kR], Br[kR], Cr[kR];
    f2_t A2[kP ? kG : 1], B2[kP ? kG : 1], C2[kP ? kG : 1];
    int c0;                                          // candidates c0 .. c0 + kR - 1
};

// Row constants of one consumer thread.  Rows past the owner's end carry n = 2^24 so that
// their k falls outside every trace; nf > 0 keeps sqrt(n^2 + Cq) + n > 0.
struct RowConst {
    int n;
    float nf, nsq;
    f2_t nf2, nsq2;
};

__device__ __forceinline__ RowConst row_const(bool act, int nrow) {
    RowConst rc;
    rc.n = act ? nrow : (1 << 24);
    rc.nf = fmaxf((float)rc.n, 1e-30f);
    rc.nsq = rc.nf * rc.nf;
    rc.nf2 = pk2(rc.nf, rc.nf);
    rc.nsq2 = pk2(rc.nsq, rc.nsq);
    return rc;
}

// Start a pass: candidates c0 .. c0+kR-1 (those >= ncand are computed, then discarded).
template <int W, class CFG, class Decode>
__device__ __forceinline__ void accum_begin(Accum<W, CFG>& a, int c0, int ncand, Decode decode) {
    a.c0 = c0;
    #pragma unroll
    for (int r = 0; r < CFG::kR; ++r) {
        const int c = c0 + r;
        a.Ar[r] = a.Br[r] = a.Cr[r] = 0.f;
        if (c < ncand) decode(c, a.Ar[r], a.Br[r], a.Cr[r]);
        a.cntv[r] = 0;
    }
    #pragma unroll
    for (int g = 0; g < Accum<W, CFG>::kG; ++g) {
        if constexpr (Accum<W, CFG>::kP) {
            a.A2[g] = pk2(a.Ar[2 * g], a.Ar[2 * g + 1]);
            a.B2[g] = pk2(a.Br[2 * g], a.Br[2 * g + 1]);
            a.C2[g] = pk2(a.Cr[2 * g], a.Cr[2 * g + 1]);
            a.den2[g][0] = a.den2[g][1] = 0ull;
            #pragma unroll
            for (int j = 0; j < W; ++j) a.num2[g][j] = 0ull;
        } else {
            a.den1[g][0] = a.den1[g][1] = 0.f;
            #pragma unroll
            for (int j = 0; j < W; ++j) a.num1[g][j] = 0.f;
        }
    }
}

// Accumulate one run of traces [t0, t1) of a slot whose traces are all of one kind (FAST:
// every pair takes part).  Software pipeline: the traveltimes of trace t+1 (long MUFU
// chains) are formed while the window of trace t is accumulated.
template <bool CRS, int W, class CFG, bool FAST>
__device__ __forceinline__ void accum_run(Accum<W, CFG>& a, const TraceMeta* meta, int t0, int t1,
                                          const RowConst& rc, int zidx, const float* smf) {
    constexpr int kR = CFG::kR;
    constexpr int kG = Accum<W, CFG>::kG;
    int sI[kR];
    float sX[kR];
    bool sO[kR];
    // check-free packed runs keep each pair's fractions as one f32x2 value
    constexpr bool kX2 = FAST && CFG::kMode == kPacked;
    f2_t sX2[kX2 ? kG : 1];
    auto setup = [&](int t) {
        const TraceConst tc = trace_const(meta[t], rc.n);
        if constexpr (CFG::kMode == kPacked) {
            #pragma unroll
            for (int g = 0; g < kG; ++g) {
                if constexpr (FAST)
                    intersect_pair_fast<CRS>(a.A2[g], a.B2[g], a.C2[g], tc, rc.nf2, rc.nsq2,
                                             sI[2 * g], sI[2 * g + 1], sX2[g]);
                else
                    intersect_pair<CRS>(a.A2[g], a.B2[g], a.C2[g], tc, rc.nf2, rc.nsq2, zidx,
                                        sI[2 * g], sI[2 * g + 1], sX[2 * g], sX[2 * g + 1],
                                        sO[2 * g], sO[2 * g + 1]);
            }
        } else {
            #pragma unroll
            for (int r = 0; r < kR; ++r) {
                if constexpr (FAST)
                    intersect_one_fast<CRS>(a.Ar[r], a.Br[r], a.Cr[r], tc, rc.nf, rc.nsq, sI[r],
                                            sX[r]);
                else
                    intersect_one<CRS>(a.Ar[r], a.Br[r], a.Cr[r], tc, rc.nf, rc.nsq, zidx, sI[r],
                                       sX[r], sO[r]);
            }
        }
    };
    setup(t0);
    auto step = [&](int t, auto more) {
        int cI[kR];
        float cX[kR];
        f2_t cX2[kX2 ? kG : 1];
        #pragma unroll
        for (int r = 0; r < kR; ++r) {
            cI[r] = sI[r];
            if constexpr (!kX2) cX[r] = sX[r];
            if constexpr (!FAST) a.cntv[r] += sO[r] ? 1 : 0;
        }
        if constexpr (kX2) {
            #pragma unroll
            for (int g = 0; g < kG; ++g) cX2[g] = sX2[g];
        }
        if constexpr (decltype(more)::value) setup(t + 1);
        #pragma unroll
        for (int g = 0; g < kG; ++g) {
            if constexpr (CFG::kMode == kScalar) {
                float F[W + 1];
                #pragma unroll
                for (int j = 0; j <= W; ++j) F[j] = smf[cI[g] + j];
                #pragma unroll
                for (int j = 0; j < W; ++j) {
                    const float v = fmaf(cX[g], F[j + 1] - F[j], F[j]);
                    a.num1[g][j] += v;
                    a.den1[g][kDenChains == 2 ? (j & 1) : 0] =
                        fmaf(v, v, a.den1[g][kDenChains == 2 ? (j & 1) : 0]);
                }
            } else {
                const int ra = 2 * g, rb = 2 * g + 1;
                float FA[W + 1], FB[W + 1];
                #pragma unroll
                for (int j = 0; j <= W; ++j) { FA[j] = smf[cI[ra] + j]; FB[j] = smf[cI[rb] + j]; }
                f2_t x2;
                if constexpr (kX2) x2 = cX2[g];
                else x2 = pk2(cX[ra], cX[rb]);
                #pragma unroll
                for (int j = 0; j < W; ++j) {
                    f2_t v;
                    if constexpr (CFG::kMode == kPacked) {
                        v = fma2(x2, sub2(pk2(FA[j + 1], FB[j + 1]), pk2(FA[j], FB[j])),
                                 pk2(FA[j], FB[j]));
                    } else if constexpr (CFG::kMode == kHybridD) {
                        v = fma2(x2, pk2(FA[j + 1] - FA[j], FB[j + 1] - FB[j]), pk2(FA[j], FB[j]));
                    } else {
                        v = pk2(fmaf(cX[ra], FA[j + 1] - FA[j], FA[j]),
                                fmaf(cX[rb], FB[j + 1] - FB[j], FB[j]));
                    }
                    a.num2[g][j] = add2(a.num2[g][j], v);
                    a.den2[g][kDenChains == 2 ? (j & 1) : 0] =
                        fma2(v, v, a.den2[g][kDenChains == 2 ? (j & 1) : 0]);
                }
            }
        }
    };
    // four traces per loop iteration: the pipeline's registers rotate instead of being
    // copied, and fewer loop branches; the run's last trace sets up nothing
    #pragma unroll 4
    for (int t = t0; t < t1 - 1; ++t) step(t, std::true_type{});
    step(t1 - 1, std::false_type{});
    if constexpr (FAST) {
        #pragma unroll
        for (int r = 0; r < kR; ++r) a.cntv[r] += t1 - t0;
    }
}

// Accumulate the ntr staged traces of one slot, in list order, as runs of all-valid traces
// (bit t of allv) and checked traces.  The order of the sums is the list order whatever
// the runs, so every tile shape gives bit-identical results.
template <bool CRS, int W, class CFG>
__device__ __forceinline__ void accum_stage(Accum<W, CFG>& a, const TraceMeta* meta, int ntr,
                                            unsigned allv, const RowConst& rc,
                                            int zidx, const float* smf) {
    int t = 0;
    while (t < ntr) {
        const bool fast = (allv >> t) & 1u;
        const unsigned rest = (fast ? ~allv : allv) >> t;    // first trace of the other kind
        const int len = rest ? __ffs(rest) - 1 : 32;
        const int t1 = min(ntr, t + len);
        if (fast) accum_run<CRS, W, CFG, true>(a, meta, t, t1, rc, zidx, smf);
        else accum_run<CRS, W, CFG, false>(a, meta, t, t1, rc, zidx, smf);
        t = t1;
    }
}

// End a pass: Eq. 1 per candidate, S cube entries, running best (ties: lowest index, since
// a thread meets its candidates in increasing order).
template <int W, class CFG>
__device__ __forceinline__ void accum_end(const Accum<W, CFG>& a, int ncand, float* S_row,
                                          float& bestS, int& bestC, float& bestT) {
    #pragma unroll
    for (int r = 0; r < CFG::kR; ++r) {
        const int c = a.c0 + r;
        if (c >= ncand) continue;
        // the numerator is summed in the same chain order as the energy, so a lone
        // participating trace gives exactly S = 1
        float nu0 = 0.f, nu1 = 0.f, ac = 0.f, d0, d1;
        #pragma unroll
        for (int j = 0; j < W; ++j) {
            float v;
            if constexpr (Accum<W, CFG>::kP) {
                float lo, hi;
                up2(a.num2[r / 2][j], lo, hi);
                v = (r & 1) ? hi : lo;
            } else {
                v = a.num1[r][j];
            }
            if (kDenChains == 2 && (j & 1)) nu1 = fmaf(v, v, nu1); else nu0 = fmaf(v, v, nu0);
            ac += v;
        }
        if constexpr (Accum<W, CFG>::kP) {
            float l0, h0, l1, h1;
            up2(a.den2[r / 2][0], l0, h0);
            up2(a.den2[r / 2][1], l1, h1);
            d0 = (r & 1) ? h0 : l0;
            d1 = (r & 1) ? h1 : l1;
        } else {
            d0 = a.den1[r][0];
            d1 = a.den1[r][1];
        }
        const float nu = nu0 + nu1, dn = d0 + d1;
        const float Nf = (float)a.cntv[r];
        const float sv = (a.cntv[r] > 0 && dn > 0.f) ? nu / (Nf * dn) : 0.f;
        const float st = a.cntv[r] > 0 ? ac / (Nf * (float)W) : 0.f;
        if (S_row) S_row[c] = sv;
        if (sv > bestS) { bestS = sv; bestC = c; bestT = st; }
    }
}

// Cross-warp argmax of the row (lane) over the nwarps consumer warps' running bests.
__device__ __forceinline__ void reduce_best(const SearchSmem& sm, int nwarps, int lane, float& bs,
                                            int& bc, float& bt) {
    bs = sm.redS[0][lane];
    bt = sm.redT[0][lane];
    bc = sm.redC[0][lane];
    for (int w2 = 1; w2 < nwarps; ++w2) {
        const float sv = sm.redS[w2][lane];
        const int c = sm.redC[w2][lane];
        if (sv > bs || (sv == bs && c < bc)) { bs = sv; bc = c; bt = sm.redT[w2][lane]; }
    }
    if (bc == INT_MAX) { bc = 0; bs = 0.f; bt = 0.f; }
}

// SPLIT: the CTAs of a tile share its candidate passes (P.nsplit parts, partial argmaxes to
// P.partial, merged by merge_partials_kernel); without it the kernel ignores both fields.
template <bool CRS, int W, class CFG, bool SPLIT = false>
__global__ void __launch_bounds__(CFG::kThreads, 2) search_kernel(const SearchParams P) {
    constexpr int HW = W / 2;
    constexpr int kWarps = CFG::kWarps;
    constexpr int kR = CFG::kR;
    constexpr int kCB = CFG::kCB;
    constexpr int kConsumers = CFG::kConsumers;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SearchSmem& sm = *reinterpret_cast<SearchSmem*>(smem_raw);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // CTA = (owner, tile of 32 rows[, part of the candidate passes])
    const unsigned otile = SPLIT ? blockIdx.x / (unsigned)P.nsplit : blockIdx.x;
    const int part = SPLIT ? (int)(blockIdx.x - otile * (unsigned)P.nsplit) : 0;
    const int64_t owner = otile / P.tiles_per_owner;
    const int tile = (int)(otile - owner * P.tiles_per_owner);
    if (owner >= P.nowner) return;
    const int64_t row0 = P.out_off[owner];
    const int nrows = (int)(P.out_off[owner + 1] - row0);
    const int n0 = tile * 32;
    if (n0 >= nrows) return;                          // whole CTA: uniform
    const int64_t lbeg = P.list_off[owner];
    const int64_t M64 = P.list_off[owner + 1] - lbeg;
    const int M = M64 < 0 ? 0 : (M64 > INT_MAX ? INT_MAX : (int)M64);
    const float dt = P.dt[owner];
    const int npass_all = (P.ncand + kCB - 1) / kCB;
    const int pass_begin = SPLIT ? (int)((int64_t)part * npass_all / P.nsplit) : 0;
    const int npass = SPLIT ? (int)((int64_t)(part + 1) * npass_all / P.nsplit)
                            : npass_all;                         // passes [begin, npass)

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&sm.full[s], 32);           // the producer warp's lanes
            mbar_init(&sm.empty[s], kConsumers);  // every consumer thread
        }
        sm.abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 16) sm.zeros[threadIdx.x] = 0.f;
    __syncthreads();

    if (warp == kWarps) {
        // =============================== producer warp ================================
        const float mc = CRS ? P.m_c[owner] : 0.f;
        const int n_last = min(n0 + 31, nrows - 1);
        int pl_pass = pass_begin, pl_t = 0, pl_bpass = -1;
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
            if (pl_bpass != pl_pass) {   // candidate bounds of this pass (one per lane)
                const int c = pl_pass * kCB + lane;
                float a = 0.f, b = 0.f, cc = 0.f;
                const bool v = lane < kCB && c < P.ncand;
                if (v) decode_candidate<CRS>(P, c, a, b, cc);
                bA0 = warp_min(v ? a : FLT_MAX);  bA1 = warp_max(v ? a : -FLT_MAX);
                bB0 = warp_min(v ? b : FLT_MAX);  bB1 = warp_max(v ? b : -FLT_MAX);
                bC0 = warp_min(v ? cc : FLT_MAX); bC1 = warp_max(v ? cc : -FLT_MAX);
                pl_bpass = pl_pass;
            }
            const int first = (pl_t == 0);
            int nfit = 0;
            unsigned allv = 0u;
            const int ntr = produce_stage<CRS, HW>(
                sm.buf[slot], (int)(sm.buf[slot] - reinterpret_cast<float*>(smem_raw)),
                sm.meta[slot], &sm.full[slot], P.traces, P.trace_off, P.h, P.m,
                P.list, lbeg, M, pl_t, dt, mc, n0, n_last,
                StageBounds{bA0, bA1, bB0, bB1, bC0, bC1}, P.status, nfit, allv);
            pl_t += nfit;
            const int last = (pl_t >= M);
            if (lane == 0) sm.desc[slot] = make_desc(pl_pass, ntr, allv, first, last, 0);
            if (last) { ++pl_pass; pl_t = 0; }
            __syncwarp();
            mbar_arrive(&sm.full[slot]);
        }
        // Let every stage still in flight land before the CTA's shared memory is released.
        const int s_end = s;
        for (int s2 = max(0, s_end - kSlots + 1); s2 <= s_end; ++s2)
            mbar_wait_bounded(&sm.full[s2 % kSlots], (uint32_t)((s2 / kSlots) & 1));
        return;
    }

    // ================================ consumer warps =====================================
    const float* smf = reinterpret_cast<const float*>(smem_raw);
    const int zidx = (int)(reinterpret_cast<const float*>(sm.zeros) - smf);
    const bool act = n0 + lane < nrows;
    const RowConst rc = row_const(act, n0 + lane);
    const int n = rc.n;
    Accum<W, CFG> acc;
    acc.c0 = INT_MAX;
    // the running best of this thread's row over its candidates stays in its own entry of
    // the reduction arrays (updated once per pass), which keeps three registers free for
    // the trace loop
    sm.redS[warp][lane] = -1.f;
    sm.redC[warp][lane] = INT_MAX;
    sm.redT[warp][lane] = 0.f;
    bool aborted = false;
    auto decode = [&](int c, float& a, float& b, float& cc) { decode_candidate<CRS>(P, c, a, b, cc); };

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
        if (d.first) accum_begin(acc, d.pass * kCB + warp * kR, P.ncand, decode);
        const int ntr = min(d.ntr, kChunkT);
        // a warp whose candidates of this pass all lie past the end skips the stage
        if (ntr > 0 && acc.c0 < P.ncand)
            accum_stage<CRS, W, CFG>(acc, sm.meta[slot], ntr, d.allv, rc, zidx, smf);
        if (d.last)
            accum_end(acc, P.ncand, (P.S_cube && act) ? P.S_cube + (row0 + n) * (int64_t)P.ncand
                                                      : nullptr, sm.redS[warp][lane],
                      sm.redC[warp][lane], sm.redT[warp][lane]);
        mbar_arrive(&sm.empty[slot]);                   // this thread is done with the slot
    }

    consumer_bar(kConsumers);
    if (aborted || sm.abort_flag) return;
    if (warp == 0 && act) {
        float bs, bt;
        int bc;
        reduce_best(sm, kWarps, lane, bs, bc, bt);
        const int64_t row = row0 + n;
        if constexpr (SPLIT) {                        // one part of a split tile
            P.partial[row * P.nsplit + part] = make_float4(bs, __int_as_float(bc), bt, 0.f);
            return;
        }
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

template <bool CRS, int W, class CFG, bool SPLIT = false>
cudaError_t launch_search_w(const SearchParams& p, cudaStream_t stream) {
    static bool configured[64] = {};  // dynamic shared-memory opt-in, once per device
    const int smem = (int)sizeof(SearchSmem);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(search_kernel<CRS, W, CFG, SPLIT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    const int64_t parts = SPLIT ? p.nsplit : 1;
    const int64_t grid = p.nowner * (int64_t)p.tiles_per_owner * parts;
    if (grid <= 0) return cudaSuccess;
    if (grid > INT_MAX || parts < 1) return cudaErrorInvalidValue;
    search_kernel<CRS, W, CFG, SPLIT><<<(unsigned)grid, CFG::kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

template <bool CRS, class CFG, bool SPLIT = false>
cudaError_t launch_search_cfg(const SearchParams& p, int w, cudaStream_t stream) {
    switch (w) {
        case 1: return launch_search_w<CRS, 1, CFG, SPLIT>(p, stream);
        case 3: return launch_search_w<CRS, 3, CFG, SPLIT>(p, stream);
        case 5: return launch_search_w<CRS, 5, CFG, SPLIT>(p, stream);
        case 7: return launch_search_w<CRS, 7, CFG, SPLIT>(p, stream);
        case 9: return launch_search_w<CRS, 9, CFG, SPLIT>(p, stream);
        case 11: return launch_search_w<CRS, 11, CFG, SPLIT>(p, stream);
        case 13: return launch_search_w<CRS, 13, CFG, SPLIT>(p, stream);
        case 15: return launch_search_w<CRS, 15, CFG, SPLIT>(p, stream);
        default: return cudaErrorInvalidValue;
    }
}

// The kernel variants the autotuner chooses from (index = variant id).
using SearchV0 = SearchCfg<7, 4, kPacked>;
using SearchV1 = SearchCfg<7, 4, kScalar>;
using SearchV2 = SearchCfg<11, 2, kHybridD>;
using SearchV3 = SearchCfg<11, 2, kScalar>;
using SearchV4 = SearchCfg<15, 2, kPacked>;
using SearchV5 = SearchCfg<15, 2, kScalar>;
using SearchV6 = SearchCfg<11, 2, kHybridV>;
using SearchV7 = SearchCfg<15, 2, kHybridV>;
using SearchV8 = SearchCfg<7, 4, kHybridD>;
using SearchV9 = SearchCfg<7, 4, kHybridV>;
// 12 consumer warps and the producer: warp w runs on warp scheduler w mod 4, so each of the
// four schedulers holds three consumer warps of the CTA (the 15-warp shapes leave one with
// two and the producer, and its warps run ahead of the others' and wait)
using SearchV10 = SearchCfg<12, 2, kPacked>;
constexpr int kSearchVariants = 11;

}  // namespace seis
