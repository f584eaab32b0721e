#!/usr/bin/env python3
"""Benchmark of the semblance search on GB300 (one JSON line on rank 0).

Default workload (cmp-line): a 2-D line of 4096 CMP gathers, fold 60, half-offsets
25..3000 m, 2000 samples at 4 ms, 8 hyperbolic events with a lateral velocity gradient,
SNR 1; 201 candidates C = 4/v^2 for v in 1400..4500 m/s; window w = 11.  One step = one
cmp_semblance call over all gathers (the whole hot path: traveltime, interpolation,
semblance, argmax, stack).  The metric is interpolated trace-samples per second
(intersections x w / s); an intersection is one (gather, t0, candidate, trace) visit.
Before the timed region the autotuner picks the kernel variant on a 512-gather slice of
the same shape bucket.

Other workloads (--workload): crs-line (1024 central CMPs, aperture +-10 CMPs, fold 48,
21x21x41 grid; --centrals limits the centrals), batch (10,000 uneven CMP/CRS items in one
persistent launch; --items), refine (512 central CMPs, coarse 7x7x11 search, its 128 best
candidates per row each refined by 20 gradient-ascent steps, against the dense 41x41x81
search on --dense-centrals centrals).  The default cmp-line run also times 64 centrals of
crs-line and the refine workload and reports them as its "crs" and "refine" sub-objects.

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the
same workload (the reference arm of this build: the paper publishes no code).  Under
torchrun (N > 1) every rank processes its own line (weak scaling, no collective on the
data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W = 11
NC = 201
VMIN, VMAX = 1400.0, 4500.0
FLOPS_PER_INTERSECTION = 12 + 7 * W        # the paper's count (Eq. 2)
SM_MAX_MHZ = 2070.0
WORKLOAD = "cmp-line: 4096 gathers x fold 60 x 2000 samples @4ms, 201 C candidates, w=11"
METRIC = "semblance interpolated trace-samples/s"


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _intersections(ds, nc):
    fold = np.diff(ds["gather_off"])
    rows = np.diff(ds["out_off"])
    return int(np.sum(fold.astype(np.int64) * rows.astype(np.int64)) * nc)


def _candidates(seis, dev):
    """The 201 candidates C = 4/v^2 (v in 1400..4500 m/s), from the library's grid entry
    point: a device tensor and its host copy."""
    Cd = seis.velocity_grid(VMIN, VMAX, NC, device=dev)
    return Cd, Cd.cpu().numpy()


def _cpu_info():
    cores = os.cpu_count() or 1
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def oracle_baseline(ds, C, target_s=15.0, seed=0):
    """Time the FP64 oracle (as it stands) on a seeded sample of output rows, sized for
    roughly target_s seconds of CPU work.  Returns (trace-samples/s, info)."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    rng = np.random.default_rng(seed)
    nrows = int(ds["out_off"][-1])
    fold = int(np.diff(ds["gather_off"]).max())
    probe = np.sort(rng.choice(nrows, 64, replace=False))
    t = time.perf_counter()
    oracle.cmp_semblance(ds, C, w=W, rows=probe, want_cube=False)
    dt_probe = max(time.perf_counter() - t, 1e-4)
    per_row = dt_probe / len(probe)
    n = int(min(nrows, max(64, target_s / per_row)))
    rows = np.sort(rng.choice(nrows, n, replace=False))
    t = time.perf_counter()
    oracle.cmp_semblance(ds, C, w=W, rows=rows, want_cube=False, nthreads=threads)
    el = time.perf_counter() - t
    inter = n * len(C) * fold
    # the same oracle on one thread, on a quarter-length sample
    n1 = int(min(nrows, max(8, target_s / 4 / (per_row * threads))))
    rows1 = rows[:n1]
    t = time.perf_counter()
    oracle.cmp_semblance(ds, C, w=W, rows=rows1, want_cube=False, nthreads=1)
    el1 = time.perf_counter() - t
    oracle.cmp_semblance(ds, C, w=W, rows=rows1[:1], want_cube=False, nthreads=threads)
    cores, model = _cpu_info()
    return inter * W / el, dict(cores=threads, cpu=model, seconds=el,
                                sample=f"{n} seeded output rows of the workload "
                                       f"(x {len(C)} candidates x fold {fold}), all traces",
                                single_thread_value=n1 * len(C) * fold * W / el1,
                                single_thread_sample=f"{n1} of those rows")


def crs_oracle_baseline(ds, centrals, A, B, C, target_s=15.0):
    """Time the FP64 CRS oracle on a deterministic sample: the given central CMPs, every
    k-th output time (k chosen for about target_s seconds), all candidates.  Returns
    (trace-samples/s, info)."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    nb = oracle.aperture(ds, centrals, ds["apm"])
    nrows = int(nb[3][-1])
    probe = np.arange(0, nrows, max(1, nrows // 8))[:8]
    t = time.perf_counter()
    oracle.crs_semblance(ds, nb, A, B, C, w=W, rows=probe, nthreads=threads)
    per_row = max(time.perf_counter() - t, 1e-4) / len(probe)
    step = max(1, int(np.ceil(nrows * per_row / target_s)))
    rows = np.arange(0, nrows, step)
    t = time.perf_counter()
    oracle.crs_semblance(ds, nb, A, B, C, w=W, rows=rows, nthreads=threads)
    el = time.perf_counter() - t
    owner = np.searchsorted(nb[3], rows, side="right") - 1
    inter = int(np.sum((nb[0][owner + 1] - nb[0][owner]) * len(A) * len(B) * len(C)))
    cores, model = _cpu_info()
    return inter * W / el, dict(cores=threads, cpu=model, seconds=el,
                                sample=f"{len(centrals)} central CMPs x every {step}th output "
                                       f"time ({len(rows)} rows) x {len(A) * len(B) * len(C)} "
                                       "candidates, all aperture traces")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(mx)),
                    power_w_median=float(np.median(pw)), samples=len(sm),
                    reasons=sorted(reasons))


# the sources the search kernel is compiled from (its ncu counters stay valid while these
# are unchanged)
SEARCH_KERNEL_SOURCES = ("search_kernel.cuh", "seis_dev.cuh", "seis_internal.h",
                         "search_dispatch.cu", "search_cmp_v*.cu", "search_crs_v*.cu")


def _kernel_digest():
    csrc = os.path.join(ROOT, "paper_1907_11678_gb300", "csrc")
    h = hashlib.sha256()
    for pat in SEARCH_KERNEL_SOURCES:
        for f in sorted(glob.glob(os.path.join(csrc, pat))):
            h.update(os.path.basename(f).encode())
            h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def _profile_traffic(kernel_tag, unit_key="dram_bytes_per_gather"):
    """DRAM traffic per unit from a committed ncu summary, if it was taken on the current
    search-kernel sources (hash match); else None."""
    digest = _kernel_digest()
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.json")
    if not os.path.exists(path):
        return None, digest
    try:
        d = json.load(open(path))
    except Exception:
        return None, digest
    if d.get("kernel_sources_sha256_16") != digest:
        return None, digest
    return d.get(unit_key), digest


def _time_steps(torch, stream, fn, steps):
    """Per-step and total CUDA-event times (ms) of `steps` calls of fn on `stream`."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], t0.elapsed_time(t1)


def _max_over_ranks(torch, dist, world, dev, x):
    from paper_1907_11678_gb300 import dist as sdist
    return x if world <= 1 else sdist.max_over_ranks(x, device=dev)


# ------------------------------------------------------------------ the cmp-line workload --

def run_cmp_line(args, torch, dist, seis, synth, rank, world, dev):
    ds = synth.workload_cmp_line(seed=2 + 1000 * rank, G=args.gathers)
    Cd, C = _candidates(seis, dev)
    inter = _intersections(ds, NC)
    g = seis.to_device(ds, dev)
    # autotune on a slice in the same shape bucket (same fold, rows, candidates)
    if args.variant is None:
        sub = synth.cmp_line(min(512, args.gathers), 60, 2000, 0.004, 25.0, 3000.0, 8, 1.0,
                             seed=99, v_range=(2550.0, 3450.0), v_gradient=0.5)
        chosen, tune_ms = seis.autotune_cmp(seis.to_device(sub, dev), Cd, w=W, reps=2)
    else:                                             # fixed variant (profiling runs)
        seis.autotune_clear()
        seis.set_search_variant(args.variant)
        chosen, tune_ms = args.variant, []
    out = seis.cmp_semblance(g, Cd, w=W)              # allocate outputs once
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        seis.cmp_semblance(g, Cd, w=W, out=out)
    torch.cuda.synchronize()
    seis.device_status()

    clocks = ClockSampler(dev.index)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    kern_ms, total_ms = _time_steps(torch, stream, lambda: seis.cmp_semblance(g, Cd, w=W, out=out),
                                    args.steps)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    seis.device_status()
    total_ms = _max_over_ranks(torch, dist, world, dev, total_ms)
    ms_per_step = total_ms / args.steps

    e2e = None if args.skip_e2e else _e2e(args, ds, C, g, Cd, out, inter, world, dev, stream,
                                          torch, dist, seis)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak_tflops = sms * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    avg_kernel_s = float(np.mean(kern_ms)) / 1e3
    achieved = inter * FLOPS_PER_INTERSECTION / avg_kernel_s / 1e12
    tper, digest = _profile_traffic("search_kernel_cmp_line")
    traffic = None if tper is None else tper * g.ngathers
    workload = WORKLOAD if g.ngathers == 4096 else \
        WORKLOAD.replace("4096 gathers", f"{g.ngathers} gathers (profiling size)")
    line = {
        "metric": "CMP " + METRIC,
        "value": inter * world * W / (ms_per_step / 1e3),
        "unit": "trace-samples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded CMP line, Ricker 25 Hz events, Gaussian noise SNR 1)",
        "config": {"workload": workload, "gathers_per_gpu": g.ngathers, "fold": 60,
                   "samples": 2000, "candidates": NC, "w": W,
                   "intersections_per_step": inter * world,
                   "l2": "inputs larger than L2 (1.97 GB of traces per GPU)",
                   "parallelism": f"gathers sharded, dp{world}" if world > 1 else "1 GPU",
                   "kernel_variant": chosen,
                   "kernel_variant_name": seis.search_variants()[chosen],
                   "autotune_ms_512_gathers": [round(x, 3) for x in tune_ms]},
        "intersections_per_s": inter * world / (ms_per_step / 1e3),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": traffic,
                     "algorithmic_bytes": int(ds["traces"].nbytes + ds["h"].nbytes
                                              + 4 * 4 * int(ds["out_off"][-1])),
                     "flops_per_intersection": FLOPS_PER_INTERSECTION,
                     "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {SM_MAX_MHZ:.0f} MHz",
                     "kernel": f"search_kernel<CMP, w=11, variant {chosen}>",
                     "kernel_sources_sha256_16": digest},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the oracle runs at N=1 only
        v, info = oracle_baseline(ds, C, target_s=args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "trace-samples/s", "cores": info["cores"],
                                "kind": "oracle", "sample": info["sample"],
                                "cpu": info["cpu"], "seconds": info["seconds"],
                                "single_thread_value": info["single_thread_value"],
                                "single_thread_sample": info["single_thread_sample"]}
    return line


E2E_CHUNKS = 8


def _e2e(args, ds, C, g, Cd, out, inter, world, dev, stream, torch, dist, seis):
    """Same metric through the C ABI with the step's inputs copied from pinned host
    memory and its results copied back inside the timed region.  The gathers stream in
    E2E_CHUNKS chunks over two streams: chunk c+1's inputs travel while chunk c is searched,
    and each chunk's results return as soon as it is done."""
    G = g.ngathers
    gb = [G * c // E2E_CHUNKS for c in range(E2E_CHUNKS + 1)]
    goff = np.asarray(ds["gather_off"], np.int64)
    toff = np.asarray(ds["trace_off"], np.int64)
    ooff = np.asarray(ds["out_off"], np.int64)
    chunks = []
    for c in range(E2E_CHUNKS):
        g0, g1 = gb[c], gb[c + 1]
        t0, t1 = int(goff[g0]), int(goff[g1])
        s0, s1 = int(toff[t0]), int(toff[t1])
        r0, r1 = int(ooff[g0]), int(ooff[g1])
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        host = {"traces": pin(ds["traces"][s0:s1]), "trace_off": pin(toff[t0:t1 + 1] - s0),
                "h": pin(ds["h"][t0:t1]), "gather_off": pin(goff[g0:g1 + 1] - t0),
                "out_off": pin(ooff[g0:g1 + 1] - r0), "dt": pin(ds["dt"][g0:g1])}
        devb = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
        gc = seis.Gathers(traces=devb["traces"], trace_off=devb["trace_off"], h=devb["h"],
                          m=None, gather_off=devb["gather_off"], out_off=devb["out_off"],
                          dt=devb["dt"], ngathers=g1 - g0, ntraces=t1 - t0,
                          max_rows=g.max_rows, max_trace_samples=g.max_trace_samples,
                          rows=r1 - r0)
        outc = {k: v[r0:r1] for k, v in out.items()}
        outh = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in outc.items()}
        chunks.append((host, devb, gc, outc, outh))
    Ch = torch.from_numpy(C).pin_memory()
    Cd2 = torch.empty_like(Cd)
    h2d = sum(v.numel() * v.element_size() for ch in chunks for v in ch[0].values()) + Ch.numel() * 4
    d2h = sum(v.numel() * v.element_size() for v in out.values())
    copy = torch.cuda.Stream(device=dev)

    def e2e_step():
        copy.wait_stream(stream)                  # the previous step's readers are done
        with torch.cuda.stream(copy):
            Cd2.copy_(Ch, non_blocking=True)
        ready = []
        for host, devb, _, _, _ in chunks:        # all inputs, in chunk order
            with torch.cuda.stream(copy):
                for k in host:
                    devb[k].copy_(host[k], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy)
            ready.append(ev)
        for (_, _, gc, outc, outh), ev in zip(chunks, ready):
            stream.wait_event(ev)
            seis.cmp_semblance(gc, Cd2, w=W, out=outc, stream=stream)
            done = torch.cuda.Event()
            done.record(stream)
            copy.wait_event(done)
            with torch.cuda.stream(copy):
                for k in outc:
                    outh[k].copy_(outc[k], non_blocking=True)
        stream.wait_stream(copy)                  # the step ends when its results are home
    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    _, total = _time_steps(torch, stream, e2e_step, args.steps)
    e2e_ms = _max_over_ranks(torch, dist, world, dev, total / args.steps)
    got = np.concatenate([ch[4]["best_idx"].numpy() for ch in chunks])
    assert np.array_equal(got, out["best_idx"].cpu().numpy())
    return {"value": inter * world * W / (e2e_ms / 1e3), "unit": "trace-samples/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": e2e_ms, "chunks": E2E_CHUNKS}


# ------------------------------------------------------------------ the other workloads ----

def _crs_grids(seis, dev, synth, nA, nB, nC):
    """The CRS A, B, C axes over the ranges of the synthetic model (library grid entry point)."""
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    return (seis.linear_grid(alo, ahi, nA, device=dev), seis.linear_grid(blo, bhi, nB, device=dev),
            seis.linear_grid(clo, chi, nC, device=dev))


def _simple_line(metric, value, ms, args, world, config, extra=None, clk=None, launches=None):
    d = {"metric": metric, "value": value, "unit": "trace-samples/s", "n_gpus": world,
         "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
         "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
         "config": config, "e2e": None, "gpu_launches": launches, "clocks": clk}
    if extra:
        d.update(extra)
    return d


def run_crs_line(args, torch, dist, seis, synth, rank, world, dev):
    ds = synth.workload_crs_line(seed=3 + 1000 * rank)
    g = seis.to_device(ds, dev)
    central = ds["central"][:args.centrals]
    ap = seis.crs_aperture(g, central, ds["apm"])
    A, B, C = _crs_grids(seis, dev, synth, 21, 21, 41)
    inter = int((ap.nbr_off[1:] - ap.nbr_off[:-1]).sum().item()) * 1500 * 21 * 21 * 41
    # autotune on a 6-central slice in the same shape bucket (candidates, rows, fold): 282
    # CTAs, about one wave with two CTAs on most SMs, as in the full run
    if args.variant is None:
        apt = seis.crs_aperture(g, ds["central"][:6], ds["apm"])
        chosen, tune_ms = seis.autotune_crs(g, apt, A, B, C, w=W, reps=1)
    else:
        seis.autotune_clear()
        seis.set_search_variant(args.variant)
        chosen, tune_ms = args.variant, []
    split = getattr(args, "split", False)
    seis.crs_semblance(g, ap, A, B, C, w=W, split=split)
    for _ in range(args.warmup - 1):
        seis.crs_semblance(g, ap, A, B, C, w=W, split=split)
    torch.cuda.synchronize()
    seis.device_status()
    clocks = ClockSampler(dev.index)
    clocks.start()
    kern, total = _time_steps(torch, torch.cuda.current_stream(),
                              lambda: seis.crs_semblance(g, ap, A, B, C, w=W, split=split),
                              args.steps)
    clk = clocks.stop()
    ms = _max_over_ranks(torch, dist, world, dev, total / args.steps)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    ach = inter * FLOPS_PER_INTERSECTION / (np.mean(kern) / 1e3) / 1e12
    # unique bytes: the traces of every CMP some aperture reaches, read once, plus 6 output
    # values per row; DRAM traffic scaled from the committed capture by the CMPs read
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        host = lambda t: t.cpu().numpy().astype(np.float64)
        v, info = crs_oracle_baseline(ds, ds["central"][::128][:8], host(A), host(B), host(C),
                                      target_s=args.cpu_seconds)
        cpu = {"value": v, "unit": "trace-samples/s", "kind": "oracle", **info}
    tr_ids = ap.nbr_trace[:int(ap.nbr_off[-1])].cpu().numpy()
    cmps = np.unique(np.searchsorted(ds["gather_off"], tr_ids, side="right") - 1)
    cmp_bytes = int(sum(ds["trace_off"][ds["gather_off"][c + 1]] - ds["trace_off"][ds["gather_off"][c]]
                        for c in cmps)) * 4
    alg_bytes = cmp_bytes + ap.rows * 6 * 4
    tper, digest = _profile_traffic("search_kernel_crs_line", "dram_bytes_per_cmp_read")
    traffic = None if tper is None else tper * len(cmps)
    return _simple_line("CRS " + METRIC, inter * world * W / (ms / 1e3), ms, args, world,
                        {"workload": f"crs-line: {len(central)} central CMPs of 1024, aperture "
                                     "+-10 CMPs (1008 traces), 1500 samples @4ms, 21x21x41, w=11",
                         "intersections_per_step": inter * world, "kernel_variant": chosen,
                         "kernel_variant_name": seis.search_variants()[chosen],
                         "autotune_ms_6_centrals": [round(x, 3) for x in tune_ms],
                         "split_candidates_over_ctas": bool(split)},
                        {"intersections_per_s": inter * world / (ms / 1e3),
                         "roofline": {"bound": "alu", "achieved": ach, "peak": peak,
                                      "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
                                      "algorithmic_bytes": alg_bytes,
                                      "flops_per_intersection": FLOPS_PER_INTERSECTION,
                                      "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x "
                                                    f"{SM_MAX_MHZ:g} MHz",
                                      "kernel": f"search_kernel<CRS, w=11, variant {chosen}>",
                                      "kernel_sources_sha256_16": digest},
                         "cpu_baseline": cpu},
                        clk, args.steps)


def run_batch(args, torch, dist, seis, synth, rank, world, dev):
    ds, items, A, B, C = synth.batch_workload(n_items=args.items, seed=4 + 1000 * rank)
    g = seis.to_device(ds, dev)
    b = seis.batch_to_device(items, A, B, C, ds["out_rows"], dev)
    ncand = np.where(items["kind"] == 1, items["nA"] * items["nB"] * items["nC"], items["nC"])
    inter = int(np.sum((items["trace_end"] - items["trace_begin"]) * items["rows"].astype(np.int64)
                       * ncand))
    # autotune the batch kernel's tile shape on every 10th item (same size mix)
    if args.variant is None:
        bsub = seis.batch_to_device(items[::10], A, B, C, ds["out_rows"], dev)
        chosen, tune_ms = seis.autotune_batch(g, bsub, w=W, reps=1)
        del bsub
    else:
        seis.autotune_clear()
        seis.set_search_variant(args.variant)
        chosen, tune_ms = args.variant, []
    out = seis.batch_semblance(g, b, w=W, mode=0)
    torch.cuda.synchronize()
    seis.device_status()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        seis.batch_semblance(g, b, w=W, mode=0, out=out)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    _, total = _time_steps(torch, torch.cuda.current_stream(), graph.replay, args.steps)
    clk = clocks.stop()
    ms = _max_over_ranks(torch, dist, world, dev, total / args.steps)
    # the comparison: one launch per item (same kernel, one step, host wall clock)
    t0 = time.perf_counter()
    seis.batch_semblance(g, b, w=W, mode=1, out=out)
    torch.cuda.synchronize()
    per_item_ms = (time.perf_counter() - t0) * 1e3
    seis.device_status()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    # the replayed graph is the task-table kernel (one CTA) and the persistent batch kernel:
    # the step time is the batch kernel's to within the setup's few microseconds
    ach = inter * FLOPS_PER_INTERSECTION / (total / args.steps / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None,
            "flops_per_intersection": FLOPS_PER_INTERSECTION,
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {SM_MAX_MHZ:g} MHz",
            "kernel": f"batch_kernel<w=11, variant {chosen}> (one persistent launch per step)"}
    return _simple_line("batched CMP+CRS " + METRIC, inter * world * W / (ms / 1e3), ms, args,
                        world,
                        {"workload": f"batch: {args.items} items (CMP p=0.5: 101-201 C; CRS "
                                     "11x11x21), fold 8-120, 1000-4000 samples @2/4 ms, w=11, "
                                     "one persistent launch in a CUDA graph",
                         "intersections_per_step": inter * world, "kernel_variant": chosen,
                         "kernel_variant_name": seis.search_variants()[chosen],
                         "autotune_ms_every_10th_item": [round(x, 3) for x in tune_ms]},
                        {"intersections_per_s": inter * world / (ms / 1e3),
                         "roofline": roof,
                         "one_launch_per_item_ms": per_item_ms,
                         "speedup_vs_one_launch_per_item": per_item_ms / ms},
                        clk, 2 * args.steps)


def run_refine(args, torch, dist, seis, synth, rank, world, dev):
    """Coarse 7x7x11 search, its nstart best candidates per row as starts, 20 projected BFGS
    steps from each (adjoint kernel), best kept -- against the dense 41x41x81 search timed on
    whole waves of CTAs.  Each part is timed with CUDA events on the launching stream."""
    ds = synth.workload_crs_refine(seed=5 + 1000 * rank)
    g = seis.to_device(ds, dev)
    central = ds["central"][:args.centrals]          # all 512 unless profiling a slice
    ap = seis.crs_aperture(g, central, ds["apm"])
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    lo, hi = [alo, blo, clo], [ahi, bhi, chi]
    ncA, ncB, ncC = (int(v) for v in args.coarse.split(","))
    A7, B7, C11 = _crs_grids(seis, dev, synth, ncA, ncB, ncC)
    nstart, steps = args.starts, args.refine_steps
    local_max = args.start_rule == "localmax"
    ws = torch.empty(seis.load_library().seis_refine_multi_workspace_size(ap.rows) + 256,
                     dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    marks = []

    def refine_all(record=False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)] if record else None
        coarse = seis.crs_semblance(g, ap, A7, B7, C11, w=W, want_cube=True)
        starts = seis.crs_top_starts(coarse["S"], A7, B7, C11, nstart, local_max=local_max)
        if record:
            ev[0].record(stream)
        ref = seis.crs_refine_multi(g, ap, starts, lo, hi, steps=steps, step0=0.05, w=W,
                                    workspace=ws)
        if record:
            ev[1].record(stream)
            marks.append(ev)
        return coarse, ref
    for _ in range(args.warmup):
        refine_all()
    torch.cuda.synchronize()
    seis.device_status()
    clocks = ClockSampler(dev.index)
    clocks.start()
    kern, total = _time_steps(torch, stream, lambda: refine_all(record=True), args.steps)
    clk = clocks.stop()
    seis.device_status()
    refine_ms = total / args.steps
    multi_ms = float(np.mean([a.elapsed_time(b) for a, b in marks]))
    search_ms = float(np.mean(kern)) - multi_ms       # coarse search + start selection
    coarse, ref = refine_all()
    one = seis.crs_refine(g, ap, coarse["best_ABC"], lo, hi, steps=steps, step0=0.05, w=W)
    # a second, smaller start count timed the same way (quality against time)
    few = None
    if args.refine_also_starts and args.refine_also_starts != nstart:
        k2 = args.refine_also_starts

        def refine_few():
            c2 = seis.crs_semblance(g, ap, A7, B7, C11, w=W, want_cube=True)
            st2 = seis.crs_top_starts(c2["S"], A7, B7, C11, k2, local_max=local_max)
            return seis.crs_refine_multi(g, ap, st2, lo, hi, steps=steps, step0=0.05, w=W,
                                         workspace=ws)
        refine_few()
        torch.cuda.synchronize()
        _, tot2 = _time_steps(torch, stream, refine_few, args.steps)
        few = (k2, tot2 / args.steps, refine_few())
    # the other start rule, untimed, for comparison (optional: it repeats the refinement)
    other = None
    if args.compare_start_rules:
        other = seis.crs_refine_multi(g, ap, seis.crs_top_starts(coarse["S"], A7, B7, C11, nstart,
                                                                 local_max=not local_max),
                                      lo, hi, steps=steps, step0=0.05, w=W, workspace=ws)
    # the dense 41x41x81 search on a slice of centrals, timed and extrapolated
    nd = min(args.dense_centrals, len(central))
    apd = seis.crs_aperture(g, central[:nd], ds["apm"])
    A41, B41, C81 = _crs_grids(seis, dev, synth, 41, 41, 81)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    dense = seis.crs_semblance(g, apd, A41, B41, C81, w=W)
    e1.record()
    torch.cuda.synchronize()
    seis.device_status()
    dense_ms_slice = e0.elapsed_time(e1)
    dense_ms = dense_ms_slice * len(central) / nd
    rows_d = apd.rows
    S_dense = dense["best_S"].cpu().numpy()
    bins = [0.0, 0.005, 0.02, 0.1, 1.01]

    def quality(S):
        gap = S_dense - S[:rows_d].cpu().numpy()
        ok = gap <= 1e-3
        per = {f"S_dense in [{a:g},{min(b, 1.0):g})":
               {"rows": int(((S_dense >= a) & (S_dense < b)).sum()),
                "within_1e-3": float(ok[(S_dense >= a) & (S_dense < b)].mean())}
               for a, b in zip(bins[:-1], bins[1:])}
        return {"rows_within_1e-3_of_dense": float(ok.mean()),
                "rows_above_dense": float(np.mean(gap < 0)),
                "median_S_refined_minus_dense": float(np.median(-gap)), "by_S_dense": per}
    trace_rows = int((ap.nbr_off[1:] - ap.nbr_off[:-1]).sum().item()) * 2000
    inter_coarse = trace_rows * ncA * ncB * ncC
    inter_eval = trace_rows * nstart * (steps + 1)
    inter_refine = inter_coarse + inter_eval
    launches = 2 + nstart * (2 * steps + 3)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    flops_eval = FLOPS_PER_INTERSECTION + 8 * W      # evaluation + adjoint (4 FMAs per sample)
    ach_eval = inter_eval * flops_eval / (multi_ms / 1e3) / 1e12
    ach_search = inter_coarse * FLOPS_PER_INTERSECTION / (search_ms / 1e3) / 1e12
    return _simple_line("CRS refine " + METRIC, inter_refine * W / (refine_ms / 1e3), refine_ms,
                        args, world,
                        {"workload": f"refine: {len(central)} central CMPs of 512, aperture +-8 "
                                     "CMPs (816 traces), "
                                     f"2000 samples @4ms; coarse {ncA}x{ncB}x{ncC}, {nstart} "
                                     f"starts per row ({'the best local maxima of the coarse cube' if local_max else 'the best coarse candidates'}) "
                                     f"each refined by {steps} projected BFGS gradient-ascent "
                                     "steps, best kept; vs dense 41x41x81",
                         "starts": nstart, "start_rule": args.start_rule, "steps": steps,
                         "dense_centrals_timed": nd,
                         "dense_ctas": int(nd * ((2000 + 31) // 32)),
                         "resident_cta_slots": 2 * sms},
                        {"refine_ms": refine_ms, "coarse_search_ms": search_ms,
                         "refine_multi_ms": multi_ms,
                         "dense_ms_extrapolated": dense_ms, "dense_ms_slice": dense_ms_slice,
                         "speedup_refine_vs_dense": dense_ms / refine_ms,
                         **quality(ref["S"]),
                         "one_start (untimed, for comparison)": quality(one["S"]),
                         **({f"start rule {'top' if local_max else 'localmax'} (untimed, for comparison)":
                             quality(other["S"])} if other is not None else {}),
                         **({f"{few[0]} starts (timed the same way)":
                             {"refine_ms": few[1], "speedup_refine_vs_dense": dense_ms / few[1],
                              **quality(few[2]["S"])}} if few is not None else {}),
                         "mean_S_gain_over_coarse": float((ref["S"] - coarse["best_S"]).mean()),
                         "roofline": {"bound": "alu", "kernel": "eval_kernel<CRS, w=11, adjoint>",
                                      "achieved": ach_eval, "peak": peak, "unit": "TFLOP/s",
                                      "frac": ach_eval / peak, "traffic": None,
                                      "flops_per_evaluation": flops_eval,
                                      "evaluation_intersections_per_step": inter_eval,
                                      "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x "
                                                    f"{SM_MAX_MHZ:g} MHz",
                                      "coarse_search_frac": ach_search / peak}},
                        clk, launches)


def run_t0win(args, torch, dist, seis, synth, rank, world, dev):
    """The window over neighbouring output times (one interpolation per intersection)
    against the paper's window along each trace, on the cmp-line workload."""
    ds = synth.workload_cmp_line(seed=2 + 1000 * rank, G=args.gathers)
    Cd, C = _candidates(seis, dev)
    inter = _intersections(ds, NC)
    g = seis.to_device(ds, dev)
    stream = torch.cuda.current_stream()
    # the paper's window runs with the variant the autotuner picks for this shape
    sub = synth.cmp_line(min(512, args.gathers), 60, 2000, 0.004, 25.0, 3000.0, 8, 1.0,
                         seed=99, v_range=(2550.0, 3450.0), v_gradient=0.5)
    seis.autotune_cmp(seis.to_device(sub, dev), Cd, w=W, reps=1)
    out_t = seis.cmp_semblance_t0win(g, Cd, w=W)
    out_p = seis.cmp_semblance(g, Cd, w=W)
    for _ in range(args.warmup):
        seis.cmp_semblance_t0win(g, Cd, w=W, out=out_t)
    torch.cuda.synchronize()
    seis.device_status()
    clocks = ClockSampler(dev.index)
    clocks.start()
    kern, total = _time_steps(torch, stream, lambda: seis.cmp_semblance_t0win(g, Cd, w=W, out=out_t),
                              args.steps)
    clk = clocks.stop()
    ms = total / args.steps
    _, total_p = _time_steps(torch, stream, lambda: seis.cmp_semblance(g, Cd, w=W, out=out_p), 2)
    total_p /= 2
    seis.device_status()
    same = (out_t["best_idx"] == out_p["best_idx"]).float().mean().item()
    near = ((out_t["best_idx"] - out_p["best_idx"]).abs() <= 2).float().mean().item()
    strong = out_p["best_S"] >= 0.1
    same_strong = ((out_t["best_idx"] == out_p["best_idx"]) & strong).sum().item() / max(
        1, strong.sum().item())
    ngathers = g.ngathers
    del g, out_t, out_p
    # CRS: 64 central CMPs of the crs-line workload, 21 x 21 x 41
    dc = synth.workload_crs_line(seed=3 + 1000 * rank)
    gc = seis.to_device(dc, dev)
    ap = seis.crs_aperture(gc, dc["central"][:64], dc["apm"])
    A, B, Cc = _crs_grids(seis, dev, synth, 21, 21, 41)
    apt = seis.crs_aperture(gc, dc["central"][:6], dc["apm"])
    seis.autotune_crs(gc, apt, A, B, Cc, w=W, reps=1)
    seis.crs_semblance_t0win(gc, ap, A, B, Cc, w=W)
    torch.cuda.synchronize()
    _, crs_t = _time_steps(torch, stream, lambda: seis.crs_semblance_t0win(gc, ap, A, B, Cc, w=W), 2)
    _, crs_p = _time_steps(torch, stream, lambda: seis.crs_semblance(gc, ap, A, B, Cc, w=W), 1)
    seis.device_status()
    crs_inter = int((ap.nbr_off[1:] - ap.nbr_off[:-1]).sum().item()) * 1500 * 21 * 21 * 41
    return _simple_line("CMP t0-window semblance intersections/s", inter * world / (ms / 1e3),
                        ms, args, world,
                        {"workload": f"cmp-line: {ngathers} gathers x fold 60 x 2000 samples "
                                     "@4ms, 201 C, w=11; window over neighbouring output times "
                                     "(one interpolated sample per intersection)",
                         "intersections_per_step": inter * world},
                        {"unit": "intersections/s",
                         "paper_window_ms": total_p, "speedup_vs_paper_window": total_p / ms,
                         "rows_same_pick_as_paper_window": same,
                         "rows_pick_within_2_candidates": near,
                         "rows_same_pick_where_paper_S_ge_0.1": same_strong,
                         "crs_64_centrals": {"t0_window_ms": crs_t / 2, "paper_window_ms": crs_p,
                                             "speedup": crs_p / (crs_t / 2),
                                             "t0_window_intersections_per_s":
                                                 crs_inter / (crs_t / 2e3)}},
                        clk, args.steps + 3)


def run_pragmatic(args, torch, dist, seis, synth, rank, world, dev):
    """The CRS operator by a central-CMP C search and a zero-offset (A, B) search, against
    the dense 21 x 21 x 41 search on the same centrals (crs-line workload)."""
    ds = synth.workload_crs_line(seed=3 + 1000 * rank)
    g = seis.to_device(ds, dev)
    ncen = min(args.centrals, 64)
    central = ds["central"][:ncen]
    ap = seis.crs_aperture(g, central, ds["apm"])
    ap_c = seis.crs_aperture(g, central, 0.0)
    ap_z = seis.crs_aperture(g, central, ds["apm"], hmax=0.0)
    (alo, ahi), (blo, bhi), _ = synth.crs_ranges()
    lo, hi = [alo, blo, synth.crs_ranges()[2][0]], [ahi, bhi, synth.crs_ranges()[2][1]]
    A, B, C = _crs_grids(seis, dev, synth, 21, 21, 41)
    ws = torch.empty(seis.load_library().seis_pragmatic_workspace_size(ap.rows) + 256,
                     dtype=torch.uint8, device=dev)
    prag = lambda: seis.crs_pragmatic(g, ap, ap_c, ap_z, A, B, C, float(C[0]), w=W, workspace=ws)
    for _ in range(args.warmup):
        prag()
    torch.cuda.synchronize()
    seis.device_status()
    clocks = ClockSampler(dev.index)
    clocks.start()
    _, total = _time_steps(torch, torch.cuda.current_stream(), prag, args.steps)
    clk = clocks.stop()
    ms = total / args.steps
    res = prag()
    # the same start refined by 20 projected BFGS steps (untimed above; timed once here)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref = seis.crs_refine(g, ap, res["theta"], lo, hi, steps=20, step0=0.05, w=W)
    torch.cuda.synchronize()
    refine_ms = (time.perf_counter() - t0) * 1e3
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    dense = seis.crs_semblance(g, ap, A, B, C, w=W)
    e1.record()
    torch.cuda.synchronize()
    seis.device_status()
    dense_ms = e0.elapsed_time(e1)
    Sd = dense["best_S"].cpu().numpy()

    def quality(S):
        gap = Sd - S.cpu().numpy()
        ev = Sd >= 0.1
        return {"rows_within_1e-3_of_dense": float(np.mean(gap <= 1e-3)),
                "event_rows_within_1e-3 (S_dense >= 0.1)": float(np.mean(gap[ev] <= 1e-3)),
                "median_S_minus_dense": float(np.median(-gap))}
    nz = int(ap_z.nbr_off[1] - ap_z.nbr_off[0])
    return _simple_line("CRS pragmatic (C on the central CMP, A and B on zero offsets) time",
                        ms, ms, args, world,
                        {"workload": f"crs-line: {ncen} central CMPs, aperture +-10 CMPs (1008 "
                                     f"traces; {nz} zero-offset), 1500 samples @4ms; 41 C on "
                                     "the central CMP, 21 x 21 (A, B) on zero offsets, then S "
                                     "over the full aperture; vs dense 21x21x41"},
                        {"unit": "ms", "higher_is_better": False,
                         "dense_ms": dense_ms, "speedup_vs_dense": dense_ms / ms,
                         **quality(res["S"]),
                         "then_20_refine_steps": {"extra_ms": refine_ms,
                                                  "speedup_vs_dense": dense_ms / (ms + refine_ms),
                                                  **quality(ref["S"])}},
                        clk, 5 * args.steps)


# The paper's Table 1 shapes: (shape, CMP gathers, CRS central CMPs, CRS aperture in CMPs
# per side).  Gathers are chosen so that each CMP input is about 1 GB (larger than L2);
# the CRS apertures hold 1260 (fold 60) or 5000 (fold 1000) traces, and the centrals give
# CTA counts (centrals x tiles of 32 rows) just under a whole number of waves of the 304
# resident CTA slots (1152 = 3.8 waves, 884 = 2.9, 288 = 0.95, 572 = 1.9).
PAPER_RUNS = [("data1/data2", 8192, 64, 10), ("data3/data4", 2048, 17, 10),
              ("data5/data6", 512, 16, 2), ("data7/data8", 128, 11, 2)]


def run_paper(args, torch, dist, seis, synth, rank, world, dev):
    Cd, C = _candidates(seis, dev)
    A, B, Cc = _crs_grids(seis, dev, synth, 21, 21, 41)
    ncrs = 21 * 21 * 41
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    stream = torch.cuda.current_stream()
    entries = []
    clocks = ClockSampler(dev.index)
    clocks.start()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        seis.device_status()
        kern, total = _time_steps(torch, stream, fn, args.steps)
        seis.device_status()
        return float(np.mean(kern)), total / args.steps

    def entry(shape, method, units, fold, ns, ncand, inter, kern_ms, ms, chosen):
        return {"dataset": shape, "method": method, **units, "fold": fold, "samples": ns,
                "candidates": ncand, "intersections": inter, "ms": ms,
                "intersections_per_s": inter / (ms / 1e3),
                "trace_samples_per_s": inter * W / (ms / 1e3),
                "roofline_frac": inter * FLOPS_PER_INTERSECTION / (kern_ms / 1e3) / 1e12 / peak,
                "kernel_variant": chosen}

    for shape, G, ncen, pad in PAPER_RUNS:
        fold, ns = synth.PAPER_SHAPES[shape]
        ds = synth.workload_paper_cmp(shape, G, seed=6 + 1000 * rank)
        g = seis.to_device(ds, dev)
        if args.variant is None:
            sub = synth.workload_paper_cmp(shape, max(16, G // 8), seed=99)
            chosen, _ = seis.autotune_cmp(seis.to_device(sub, dev), Cd, w=W, reps=1)
        else:
            seis.set_search_variant(args.variant)
            chosen = args.variant
        out = seis.cmp_semblance(g, Cd, w=W)
        kern, ms = timed(lambda: seis.cmp_semblance(g, Cd, w=W, out=out))
        entries.append(entry(shape, "CMP", {"gathers": G}, fold, ns, NC, G * fold * ns * NC,
                             kern, ms, chosen))
        del g, out, ds
        ds = synth.workload_paper_crs(shape, ncen, pad, seed=7 + 1000 * rank)
        g = seis.to_device(ds, dev)
        ap = seis.crs_aperture(g, ds["central"], ds["apm"])
        if args.variant is None:
            apt = seis.crs_aperture(g, ds["central"][:2], ds["apm"])
            chosen, _ = seis.autotune_crs(g, apt, A, B, Cc, w=W, reps=1)
        inter = int((ap.nbr_off[1:] - ap.nbr_off[:-1]).sum().item()) * ns * ncrs
        kern, ms = timed(lambda: seis.crs_semblance(g, ap, A, B, Cc, w=W))
        entries.append(entry(shape, "CRS", {"central_cmps": ncen, "aperture_traces":
                                            int(ap.nbr_off[1] - ap.nbr_off[0])},
                             fold, ns, ncrs, inter, kern, ms, chosen))
        del g, ap, ds
        torch.cuda.empty_cache()
    clk = clocks.stop()
    tot_inter = sum(e["intersections"] for e in entries)
    tot_ms = sum(e["ms"] for e in entries)
    return _simple_line("paper-shaped CMP+CRS " + METRIC, tot_inter * W / (tot_ms / 1e3), tot_ms,
                        args, world,
                        {"workload": "the paper's Table 1 shapes (fold 60/1000 x 550/1650 "
                                     "samples @4 ms), CMP 201 C and CRS 21x21x41, w=11; one "
                                     "step = every dataset once",
                         "l2": "CMP inputs ~1 GB (larger than L2); CRS apertures re-read "
                               "from L2 by design"},
                        {"intersections_per_s": tot_inter / (tot_ms / 1e3),
                         "datasets": entries}, clk, len(entries) * args.steps)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1907_11678_gb300 import build as seis_build
    from paper_1907_11678_gb300 import seis, synth

    rank, world, local = _env_rank()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    seis_build.build()
    fn = {"cmp-line": run_cmp_line, "crs-line": run_crs_line, "batch": run_batch,
          "refine": run_refine, "paper": run_paper, "pragmatic": run_pragmatic,
          "t0win": run_t0win}[args.workload]
    line = fn(args, torch, dist, seis, synth, rank, world, dev)
    if args.workload == "cmp-line" and world == 1 and not args.no_secondary:
        # the CRS search and the refinement, each with its own CUDA-event time, roofline and
        # clock record, beside the CMP headline (short runs: 1 warm-up, 2 timed steps)
        for key, sub_fn, extra in (("crs", run_crs_line, {"centrals": 64}), ("refine", run_refine, {})):
            sub_args = argparse.Namespace(**{**vars(args), "steps": 2, "warmup": 1,
                                             "no_cpu_baseline": True, "variant": None, **extra})
            sub = sub_fn(sub_args, torch, dist, seis, synth, rank, world, dev)
            for k in ("n_gpus", "vs_baseline", "data", "e2e", "higher_is_better", "scaling",
                      "dtype", "cpu_baseline"):
                sub.pop(k, None)
            line[key] = sub
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import oracle
    from paper_1907_11678_gb300 import synth
    ds = synth.workload_cmp_line()
    C = oracle.velocity_grid(VMIN, VMAX, NC).astype(np.float32)
    vals, secs = [], []
    info = None
    for i in range(args.warmup + args.steps):
        v, info = oracle_baseline(ds, C, target_s=args.ref_seconds, seed=i)
        if i >= args.warmup:
            vals.append(v)
            secs.append(info["seconds"])
    value = float(np.mean(vals))
    inter_per_row = NC * 60
    line = {
        "impl": "reference",
        "metric": "CMP " + METRIC,
        "value": value,
        "unit": "trace-samples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        # a step is one bounded sample of the workload (the oracle on seeded rows), timed
        "ms_per_step": 1e3 * float(np.mean(secs)),
        "step": "one seeded sample of output rows of the cmp-line workload (all candidates and "
                "traces of each row), about --ref-seconds of oracle work, wall clock",
        "projected_full_line_ms (projection, not measured)":
            1e3 * 4096 * 2000 * inter_per_row * W / value,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded CMP line, Ricker 25 Hz events, Gaussian noise SNR 1)",
        "config": {"workload": WORKLOAD, "gathers_per_gpu": 4096, "fold": 60, "samples": 2000,
                   "candidates": NC, "w": W, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "trace-samples/s", "cores": info["cores"],
                         "kind": "oracle", "sample": info["sample"], "cpu": info["cpu"]},
        "e2e": {"value": value, "unit": "trace-samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cmp-line",
                    choices=["cmp-line", "crs-line", "batch", "refine", "paper", "pragmatic",
                             "t0win"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--gathers", type=int, default=4096,
                    help="gathers per GPU (4096 = the benchmark workload; fewer only for profiling)")
    ap.add_argument("--centrals", type=int, default=1024, help="crs-line: central CMPs")
    ap.add_argument("--items", type=int, default=10000, help="batch: items")
    ap.add_argument("--dense-centrals", type=int, default=24,
                    help="refine: dense-grid slice (24 x 63 tiles = 4.97 waves of 304 CTAs)")
    ap.add_argument("--starts", type=int, default=128, help="refine: coarse starts per row")
    ap.add_argument("--refine-also-starts", type=int, default=16,
                    help="refine: also time this start count (0: no)")
    ap.add_argument("--compare-start-rules", action="store_true",
                    help="refine: also report the other start rule's quality (untimed)")
    ap.add_argument("--coarse", default="7,7,11", help="refine: coarse grid nA,nB,nC")
    ap.add_argument("--refine-steps", type=int, default=20, help="refine: BFGS trials per start")
    ap.add_argument("--start-rule", default="top", choices=["localmax", "top"],
                    help="refine: starts at the coarse cube's best local maxima or its best "
                         "candidates")
    ap.add_argument("--skip-e2e", action="store_true", help="profiling runs only")
    ap.add_argument("--split", action="store_true",
                    help="crs-line: spread each tile's candidates over several CTAs when the "
                         "centrals do not fill the GPU (crs_semblance_ws)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="cmp-line: leave out the crs and refine sub-objects")
    ap.add_argument("--variant", type=int, default=None,
                    help="force a search kernel variant instead of autotuning (profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
