// batch_kernel.cuh -- one persistent launch over thousands of uneven CMP gathers and CRS
// supergathers (seis_batch_semblance).
//
// Same arithmetic as the search kernel (Eq. 1, Algorithm 1, Section 3.2 argmax and stack;
// CMP items run through the CRS traveltime with dm = 0 and A = B = 0, which reproduces the
// CMP traveltime bit for bit).  Work unit = task = (item, tile of 32 output rows).  The
// producer warp of each resident CTA claims tasks from a device counter (the task table is
// ordered as the items, so callers put costly items first) and streams their stages through
// the shared-memory ring without a break at task boundaries; the consumer warps finish a
// task's argmax when its last pass ends and go on with the next task's stages.
#pragma once
#include "search_kernel.cuh"

namespace seis {

struct ItemView {
    int64_t lbeg;
    int M;
    int64_t row0;
    int nrows;
    float dt, mc;
    int kind, a_off, nA, b_off, nB, c_off, nC, ncand;
};

__device__ __forceinline__ ItemView load_item(const BatchParams& P, int64_t i) {
    const seis_batch_item it = P.items[i];
    ItemView v;
    v.lbeg = it.trace_begin;
    v.M = (int)(it.trace_end - it.trace_begin);
    v.row0 = it.out_begin;
    v.nrows = it.rows;
    v.dt = it.dt;
    v.mc = it.m_c;
    v.kind = it.kind;
    v.a_off = it.a_off;
    v.nA = it.kind ? it.nA : 1;
    v.b_off = it.b_off;
    v.nB = it.kind ? it.nB : 1;
    v.c_off = it.c_off;
    v.nC = it.nC;
    v.ncand = v.nA * v.nB * v.nC;
    return v;
}

__device__ __forceinline__ void decode_item(const BatchParams& P, const ItemView& v, int c,
                                            float& a, float& b, float& cc) {
    const int nbc = v.nB * v.nC;
    const int ia = c / nbc;
    const int rem = c - ia * nbc;
    const int ib = rem / v.nC;
    const int ic = rem - ib * v.nC;
    a = v.kind ? P.poolA[v.a_off + ia] : 0.f;
    b = v.kind ? P.poolB[v.b_off + ib] : 0.f;
    cc = P.poolC[v.c_off + ic];
}

// Largest item i in [lo, hi) with task_off[i] <= t (task_off non-decreasing), found by the
// whole warp: each round the 32 lanes probe 32 evenly spaced entries of the interval at
// once, so a table of N items takes about log32(N) rounds of loads instead of log2(N)
// dependent ones.  Every lane returns the same item.
__device__ __forceinline__ int64_t item_of_task_warp(const int64_t* task_off, int64_t lo,
                                                     int64_t hi, int64_t t) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 1) {
        const int64_t span = hi - lo;
        const int64_t step = (span + 31) / 32;            // probes lo + lane * step
        const int64_t probe = lo + (int64_t)lane * step;
        const bool le = probe < hi && task_off[probe] <= t;
        const unsigned m = __ballot_sync(kFull, le);     // a prefix of the lanes (lane 0 set)
        const int k = 31 - __clz(m);                     // last probe with task_off <= t
        const int64_t nlo = lo + (int64_t)k * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    return lo;
}

// The search kernel's shared memory plus, per ring slot, the candidates of the pass that
// the slot's stage starts: the producer has them in registers when it bounds the pass, so
// consumers take them from here (and the task's sizes from the stage descriptor) instead of
// loading the item table and the candidate pools from global memory at every pass (for
// small-fold items a pass is a single stage of a few traces, and that latency would stall
// every warp once per stage).  The consumers keep no per-task state in registers beyond
// their row's constants: everything else comes with each stage.
struct BatchSmem {
    SearchSmem s;
    float4 cand[kSlots][32];     // (A, B, C, -) of candidates pass * kCB + lane
    ItemView item;               // the producer's current item (read back as needed, which
                                 // keeps the producer warp's registers few)
};

template <int W, class CFG>
__global__ void __launch_bounds__(CFG::kThreads, 2) batch_kernel(const BatchParams P) {
    constexpr int HW = W / 2;
    constexpr int kWarps = CFG::kWarps;
    constexpr int kR = CFG::kR;
    constexpr int kCB = CFG::kCB;
    constexpr int kConsumers = CFG::kConsumers;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BatchSmem& bsm = *reinterpret_cast<BatchSmem*>(smem_raw);
    SearchSmem& sm = bsm.s;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t t_begin = P.task_off[P.item_begin];
    const int64_t t_end = P.task_off[P.item_end];

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&sm.full[s], 32);
            mbar_init(&sm.empty[s], kConsumers);
        }
        sm.abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 16) sm.zeros[threadIdx.x] = 0.f;
    __syncthreads();

    if (warp == kWarps) {
        // =============================== producer warp ================================
        bool have = false;
        const ItemView& it = bsm.item;
        int64_t item = 0;
        // the next task is claimed one task ahead, so the atomic's latency passes while the
        // current task's stages are produced
        unsigned long long next = 0;
        if (lane == 0) next = atomicAdd(P.counter, 1ull);
        int tile = 0, n0 = 0, n_last = 0, npass = 0;
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
            bool finished = sm.abort_flag != 0;
            if (!finished && (!have || pl_pass >= npass)) {
                const unsigned long long t = __shfl_sync(kFull, next, 0);
                const int64_t tk = t_begin + (int64_t)t;
                if (tk >= t_end) {
                    finished = true;
                } else {
                    if (lane == 0) next = atomicAdd(P.counter, 1ull);
                    item = item_of_task_warp(P.task_off, P.item_begin, P.item_end, tk);
                    tile = (int)(tk - P.task_off[item]);
                    if (lane == 0) bsm.item = load_item(P, item);
                    __syncwarp();
                    n0 = tile * 32;
                    n_last = min(n0 + 31, it.nrows - 1);
                    npass = (it.ncand + kCB - 1) / kCB;
                    pl_pass = 0;
                    pl_t = 0;
                    pl_bpass = -1;
                    have = true;
                }
            }
            if (finished) {
                if (lane == 0) sm.desc[slot] = make_desc(0, 0, 0u, 0, 0, 1);
                __syncwarp();
                mbar_arrive(&sm.full[slot]);
                break;
            }
            const int first = (pl_t == 0);
            if (pl_bpass != pl_pass) {   // candidate bounds of this pass (one per lane)
                const int c = pl_pass * kCB + lane;
                float a = 0.f, b = 0.f, cc = 0.f;
                const bool v = lane < kCB && c < it.ncand;
                if (v) decode_item(P, it, c, a, b, cc);
                bA0 = warp_min(v ? a : FLT_MAX);  bA1 = warp_max(v ? a : -FLT_MAX);
                bB0 = warp_min(v ? b : FLT_MAX);  bB1 = warp_max(v ? b : -FLT_MAX);
                bC0 = warp_min(v ? cc : FLT_MAX); bC1 = warp_max(v ? cc : -FLT_MAX);
                pl_bpass = pl_pass;
                // the pass's first stage carries its candidates (released with the stage)
                bsm.cand[slot][lane] = make_float4(a, b, cc, 0.f);
            }
            int nfit = 0;
            unsigned allv = 0u;
            const int ntr = produce_stage<true, HW>(
                sm.buf[slot], (int)(sm.buf[slot] - reinterpret_cast<float*>(smem_raw)),
                sm.meta[slot], &sm.full[slot], P.traces, P.trace_off, P.h,
                it.kind ? P.m : nullptr, nullptr, it.lbeg, it.M, pl_t, it.dt, it.mc, n0, n_last,
                StageBounds{bA0, bA1, bB0, bB1, bC0, bC1}, P.status, nfit, allv);
            pl_t += nfit;
            const int last = (pl_t >= it.M);
            const int task_end = last && (pl_pass + 1 >= npass);
            if (lane == 0)
                sm.desc[slot] = make_desc(pl_pass, ntr, allv, first, last, 0, (int)item, tile,
                                          task_end, it.ncand, it.nrows);
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
    // Loops nest as task > candidate pass > stage, so a pass's accumulators live only inside
    // its loop and the task's argmax and outputs run with none of them held in registers.
    // Every pass starts with its first stage (the producer bounds and stages passes in order).
    const float* smf = reinterpret_cast<const float*>(smem_raw);
    const int zidx = (int)(reinterpret_cast<const float*>(sm.zeros) - smf);
    // the running best of this thread's row stays in its own entry of the reduction arrays
    // (updated once per pass), which keeps three registers free for the trace loop
    float& bestS = sm.redS[warp][lane];
    int& bestC = sm.redC[warp][lane];
    float& bestT = sm.redT[warp][lane];
    int s = 0;                                    // the next stage
    bool stop = false;
    while (!stop) {                               // one task per iteration
        bestS = -1.f;
        bestC = INT_MAX;
        bestT = 0.f;
        int item = 0, tile = 0, nrows = 0;
        bool task_end = false;
        while (!task_end) {                       // one candidate pass per iteration
            int slot = s % kSlots;
            if (!mbar_wait_bounded(&sm.full[slot], (uint32_t)((s / kSlots) & 1))) {
                sm.abort_flag = 1;
                record_status(P.status, kStatusTimeout);
                stop = true;
                break;
            }
            StageDesc d = sm.desc[slot];
            if (d.end) {
                stop = true;
                break;
            }
            const int ncand = d.ncand;
            const int nrow = d.tile * 32 + lane;
            const RowConst rc = row_const(nrow < d.nrows, nrow);
            const int cbase = d.pass * kCB;
            Accum<W, CFG> acc;
            const float4* cand = bsm.cand[slot];
            accum_begin(acc, cbase + warp * kR, ncand, [&](int c, float& a, float& b, float& cc) {
                const float4 v = cand[c - cbase];
                a = v.x;
                b = v.y;
                cc = v.z;
            });
            // a warp whose candidates of this pass all lie past the end skips its stages
            const bool live = acc.c0 < ncand;
            for (;;) {                            // the pass's stages
                const int ntr = min(d.ntr, kChunkT);
                if (ntr > 0 && live)
                    accum_stage<true, W, CFG>(acc, sm.meta[slot], ntr, d.allv, rc, zidx, smf);
                const bool last = d.last != 0;
                task_end = d.task_end != 0;
                item = d.item;
                tile = d.tile;
                nrows = d.nrows;
                mbar_arrive(&sm.empty[slot]);     // this thread is done with the slot
                ++s;
                if (last) break;
                slot = s % kSlots;
                if (!mbar_wait_bounded(&sm.full[slot], (uint32_t)((s / kSlots) & 1))) {
                    sm.abort_flag = 1;
                    record_status(P.status, kStatusTimeout);
                    stop = true;
                    break;
                }
                d = sm.desc[slot];
                if (d.end) {                      // the producer gave up mid-pass
                    stop = true;
                    break;
                }
            }
            if (stop) break;
            accum_end(acc, ncand, nullptr, bestS, bestC, bestT);
        }
        if (stop) break;
        // the task's last stage is done: argmax over the warps and outputs
        consumer_bar(kConsumers);
        const int nrow = tile * 32 + lane;
        if (warp == 0 && nrow < nrows) {
            const ItemView it = load_item(P, item);
            float bs, bt;
            int bc;
            reduce_best(sm, kWarps, lane, bs, bc, bt);
            float a, b, cc;
            decode_item(P, it, bc, a, b, cc);
            const int64_t row = it.row0 + nrow;
            P.best_idx[row] = bc;
            P.best_S[row] = bs;
            P.stack[row] = bt;
            if (P.best_ABC) {
                P.best_ABC[row * 3 + 0] = a;
                P.best_ABC[row * 3 + 1] = b;
                P.best_ABC[row * 3 + 2] = cc;
            }
        }
        consumer_bar(kConsumers);                 // the reduction arrays are free again
    }
}

template <int W, class CFG>
cudaError_t launch_batch_w(const BatchParams& p, int grid, cudaStream_t stream) {
    static bool configured[64] = {};
    const int smem = (int)sizeof(BatchSmem);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(batch_kernel<W, CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    if (grid <= 0) return cudaSuccess;
    batch_kernel<W, CFG><<<grid, CFG::kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

template <class CFG>
cudaError_t launch_batch_cfg(const BatchParams& p, int w, int grid, cudaStream_t s) {
    switch (w) {
        case 1: return launch_batch_w<1, CFG>(p, grid, s);
        case 3: return launch_batch_w<3, CFG>(p, grid, s);
        case 5: return launch_batch_w<5, CFG>(p, grid, s);
        case 7: return launch_batch_w<7, CFG>(p, grid, s);
        case 9: return launch_batch_w<9, CFG>(p, grid, s);
        case 11: return launch_batch_w<11, CFG>(p, grid, s);
        case 13: return launch_batch_w<13, CFG>(p, grid, s);
        case 15: return launch_batch_w<15, CFG>(p, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace seis
