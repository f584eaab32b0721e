"""Seeded synthetic seismic gathers shaped like the paper's workloads.

The paper's datasets (Table 1) are synthetic and unpublished, so every input here is
generated: Ricker-wavelet reflection events on CMP gathers with Gaussian noise at a
given signal-to-noise ratio.  This module does forward modelling only (event
traveltimes and wavelets); it contains none of the semblance search's arithmetic
(no interpolation, semblance, pick or stack), and it is the one module that feeds
both the CUDA path and the FP64 oracle.

Event traveltimes (two-way, half-offset h, midpoint m, all in SI units):
  * hyperbolic event on one CMP:      t = sqrt(t0^2 + 4 h^2 / v^2)
  * dipping plane, constant velocity: t = sqrt((t0c + 2 sin(a) (m - mc) / v)^2 + 4 cos(a)^2 h^2 / v^2)
  * point diffractor at (xd, zd):     t = (sqrt(zd^2 + (m - h - xd)^2) + sqrt(zd^2 + (m + h - xd)^2)) / v
Wavelet: Ricker r(tau) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), f = 25 Hz.
Noise: sigma_g = RMS of gather g's noise-free samples with |s| > 1e-3 * peak, divided by
SNR; seeded numpy PCG64 streams per block of gathers.

A dataset is a dict of numpy arrays:
  traces     float32 [total_samples]  trace i = traces[trace_off[i]:trace_off[i+1]]
  trace_off  int64   [ntraces+1]
  h          float32 [ntraces]        half-offset (m)
  m          float32 [ntraces]        midpoint of the trace's CDP (m)
  gather_off int64   [G+1]            traces of gather g
  out_off    int64   [G+1]            output rows of gather g (its number of samples)
  dt         float32 [G]              sampling interval (s)
"""
from __future__ import annotations

import numpy as np

RICKER_HZ = 25.0
_BLOCK = 64  # gathers per noise stream


def ricker(tau, f=RICKER_HZ):
    a = (np.pi * f * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def _layout(ns_per_trace, traces_per_gather, out_ns):
    ns_per_trace = np.asarray(ns_per_trace, np.int64)
    trace_off = np.zeros(len(ns_per_trace) + 1, np.int64)
    np.cumsum(ns_per_trace, out=trace_off[1:])
    gather_off = np.zeros(len(traces_per_gather) + 1, np.int64)
    np.cumsum(np.asarray(traces_per_gather, np.int64), out=gather_off[1:])
    out_off = np.zeros(len(out_ns) + 1, np.int64)
    np.cumsum(np.asarray(out_ns, np.int64), out=out_off[1:])
    return trace_off, gather_off, out_off


def _add_events_uniform(block, times, amps, dt, f=RICKER_HZ):
    """block: float64 [R, ns]; times: [E, R] traveltimes (s, NaN = absent); amps [E, R]."""
    R, ns = block.shape
    half = int(np.ceil(1.5 / (f * dt))) + 1  # Ricker is below 1e-9 beyond |tau| = 1.5/f
    rows = np.arange(R)
    for e in range(times.shape[0]):
        t = times[e]
        ok = np.isfinite(t)
        centre = np.where(ok, np.floor(np.where(ok, t, 0.0) / dt), -10 * half).astype(np.int64)
        for o in range(-half, half + 2):
            s = centre + o
            sel = ok & (s >= 0) & (s < ns)
            if not sel.any():
                continue
            r, ss = rows[sel], s[sel]
            block[r, ss] += amps[e, sel] * ricker(ss * dt - t[sel], f)


def _noise_sigma(block_g, snr):
    """block_g: [G, M*ns] noise-free samples; per-gather sigma."""
    peak = np.abs(block_g).max(axis=1)
    sig = np.zeros(block_g.shape[0])
    for g in range(block_g.shape[0]):
        if peak[g] <= 0:
            continue
        sel = np.abs(block_g[g]) > 1e-3 * peak[g]
        sig[g] = np.sqrt(np.mean(block_g[g][sel] ** 2)) / snr
    if (sig == 0).any() and (sig > 0).any():
        sig[sig == 0] = np.median(sig[sig > 0])
    return sig


def _render(G, M, ns, dt, snr, seed, event_fn):
    """Render G gathers of M traces x ns samples block by block (bounded memory):
    event_fn(g0, g1) -> (times [E, (g1-g0)*M], amps [E, (g1-g0)*M]); then add seeded
    Gaussian noise at the given SNR (None: no noise).  Returns float32 [G*M*ns]."""
    out = np.empty(G * M * ns, np.float32)
    L = M * ns
    for b0 in range(0, G, _BLOCK):
        b1 = min(G, b0 + _BLOCK)
        times, amps = event_fn(b0, b1)
        blk = np.zeros(((b1 - b0) * M, ns))
        if len(times):
            _add_events_uniform(blk, np.asarray(times), np.asarray(amps), dt)
        blk = blk.reshape(b1 - b0, L)
        if snr is not None and snr > 0:
            sig = _noise_sigma(blk, snr)
            rng = np.random.default_rng([seed, b0 // _BLOCK])
            blk += rng.standard_normal((b1 - b0, L), dtype=np.float32) * sig[:, None]
        out[b0 * L:b1 * L] = blk.reshape(-1)
    return out


def cmp_line(G, M, ns, dt, hmin, hmax, n_events, snr, seed, t0_range=None,
             v_range=(1500.0, 4000.0), v_gradient=0.0, dm=12.5, amp_range=(0.5, 1.0)):
    """G CMP gathers on a line (spacing dm), M traces with half-offsets evenly spaced in
    [hmin, hmax], ns samples at dt.  n_events hyperbolic events per gather with t0 ~
    U(t0_range), amplitude +-U(amp_range) and velocity v0 + v_gradient*(g - G/2), v0 ~
    U(v_range) (shared along the line)."""
    rng = np.random.default_rng(seed)
    T = ns * dt
    if t0_range is None:
        t0_range = (0.3, 0.9 * T)
    t0 = rng.uniform(*t0_range, size=n_events)
    v0 = rng.uniform(*v_range, size=n_events)
    amp = rng.uniform(*amp_range, size=n_events) * rng.choice([-1.0, 1.0], size=n_events)
    h = np.linspace(hmin, hmax, M)

    def events(g0, g1):
        g = np.arange(g0, g1)
        vel = v0[:, None] + v_gradient * (g[None, :] - G / 2.0)       # [E, gathers]
        tt = np.sqrt(t0[:, None, None] ** 2 + 4.0 * h[None, None, :] ** 2 / vel[:, :, None] ** 2)
        times = tt.reshape(n_events, (g1 - g0) * M)
        return times, np.repeat(amp[:, None], (g1 - g0) * M, axis=1)

    traces = _render(G, M, ns, dt, snr, seed, events)
    g = np.arange(G)
    trace_off, gather_off, out_off = _layout(np.full(G * M, ns), np.full(G, M), np.full(G, ns))
    return dict(traces=traces, trace_off=trace_off,
                h=np.tile(h, G).astype(np.float32),
                m=np.repeat(g * dm, M).astype(np.float32),
                gather_off=gather_off, out_off=out_off,
                dt=np.full(G, dt, np.float32),
                events=dict(t0=t0, v0=v0, amp=amp, v_gradient=v_gradient))


def crs_line(G, M, ns, dt, hmin, hmax, n_planes, n_diffractors, snr, seed, dm=12.5,
             v_range=(1500.0, 4000.0), max_dip_deg=20.0, amp_range=(0.5, 1.0)):
    """A 2-D line of G CMPs (spacing dm) with dipping planar reflectors (exact CRS form,
    B = 0) and point diffractors (double-square-root traveltime)."""
    rng = np.random.default_rng(seed)
    T = ns * dt
    mid = np.arange(G) * dm
    mcen = mid[G // 2]
    h = np.linspace(hmin, hmax, M)
    Mm = np.repeat(mid, M)
    Hh = np.tile(h, G)
    planes, diffs = [], []
    for _ in range(n_planes):
        t0c = rng.uniform(0.3, 0.85 * T)
        v = rng.uniform(*v_range)
        a = np.deg2rad(rng.uniform(-max_dip_deg, max_dip_deg))
        amp = rng.uniform(*amp_range) * rng.choice([-1.0, 1.0])
        planes.append(dict(t0c=t0c, v=v, dip=a, amp=amp, mc=mcen))
    for _ in range(n_diffractors):
        v = rng.uniform(*v_range)
        xd = rng.uniform(mid[0], mid[-1])
        zd = rng.uniform(0.3, 0.8 * T) * v / 2.0
        amp = rng.uniform(*amp_range) * rng.choice([-1.0, 1.0])
        diffs.append(dict(xd=xd, zd=zd, v=v, amp=amp))

    def events(g0, g1):
        mm = Mm[g0 * M:g1 * M]
        hh = Hh[g0 * M:g1 * M]
        times, amps = [], []
        for pl in planes:
            t0m = pl["t0c"] + 2.0 * np.sin(pl["dip"]) * (mm - mcen) / pl["v"]
            with np.errstate(invalid="ignore"):
                t = np.where(t0m > 0, np.sqrt(np.maximum(t0m, 0) ** 2
                                              + 4.0 * np.cos(pl["dip"]) ** 2 * hh ** 2 / pl["v"] ** 2),
                             np.nan)
            times.append(t); amps.append(np.full(len(mm), pl["amp"]))
        for df in diffs:
            t = (np.sqrt(df["zd"] ** 2 + (mm - hh - df["xd"]) ** 2)
                 + np.sqrt(df["zd"] ** 2 + (mm + hh - df["xd"]) ** 2)) / df["v"]
            times.append(t); amps.append(np.full(len(mm), df["amp"]))
        return times, amps

    traces = _render(G, M, ns, dt, snr, seed, events)
    trace_off, gather_off, out_off = _layout(np.full(G * M, ns), np.full(G, M), np.full(G, ns))
    return dict(traces=traces, trace_off=trace_off, h=Hh.astype(np.float32),
                m=Mm.astype(np.float32), gather_off=gather_off, out_off=out_off,
                dt=np.full(G, dt, np.float32), events=dict(planes=planes, diffractors=diffs))


# --- the workloads (shapes from the paper's problem statement; see the design notes) --

CMP_V_RANGE = (1400.0, 4500.0)


def workload_cmp_small(seed=1):
    """16 CMP gathers, fold 24, h 0..1500 m, 1000 samples at 4 ms, 5 events, SNR 2."""
    return cmp_line(16, 24, 1000, 0.004, 0.0, 1500.0, 5, 2.0, seed, t0_range=(0.3, 3.5))


def workload_cmp_line(seed=2, G=4096):
    """4096 CMP gathers on a line, fold 60, h 25..3000 m, 2000 samples at 4 ms, 8 events
    with a lateral velocity gradient of 0.5 m/s per CMP, SNR 1."""
    return cmp_line(G, 60, 2000, 0.004, 25.0, 3000.0, 8, 1.0, seed,
                    v_range=(2550.0, 3450.0), v_gradient=0.5)


def workload_crs_line(seed=3, n_central=1024, pad=10):
    """1024 central CMPs + 10 padding CMPs each side at 12.5 m, fold 48, h 0..2400 m,
    1500 samples at 4 ms; dipping planes and diffractors, SNR 2."""
    rng = np.random.default_rng(seed + 1000)
    ds = crs_line(n_central + 2 * pad, 48, 1500, 0.004, 0.0, 2400.0,
                  int(rng.integers(3, 5)), int(rng.integers(2, 4)), 2.0, seed)
    ds["central"] = np.arange(pad, pad + n_central, dtype=np.int32)
    ds["apm"] = pad * 12.5
    return ds


def workload_crs_refine(seed=5, n_central=512, pad=8):
    """512 central CMPs, aperture +-8 CMPs (100 m), fold 48, 2000 samples at 4 ms."""
    rng = np.random.default_rng(seed + 1000)
    ds = crs_line(n_central + 2 * pad, 48, 2000, 0.004, 0.0, 2400.0,
                  int(rng.integers(3, 5)), int(rng.integers(2, 4)), 2.0, seed)
    ds["central"] = np.arange(pad, pad + n_central, dtype=np.int32)
    ds["apm"] = pad * 12.5
    return ds


# The paper's Table 1 shapes (fold, samples per trace).  Its "dt" column (220 / 240) is not
# a sampling interval and is not used, so data1 and data2 (and each later pair) share one
# shape; all are sampled at 4 ms here.
PAPER_SHAPES = {"data1/data2": (60, 550), "data3/data4": (60, 1650),
                "data5/data6": (1000, 550), "data7/data8": (1000, 1650)}


def workload_paper_cmp(shape, G, seed=6):
    """G CMP gathers of a Table 1 shape on a line, h 25..3000 m, 4 ms, 6 events with a
    lateral velocity gradient of 0.5 m/s per CMP, SNR 1."""
    fold, ns = PAPER_SHAPES[shape]
    return cmp_line(G, fold, ns, 0.004, 25.0, 3000.0, 6, 1.0, seed,
                    v_range=(2550.0, 3450.0), v_gradient=0.5)


def workload_paper_crs(shape, n_central, pad, seed=7):
    """n_central central CMPs of a Table 1 shape plus pad CMPs each side at 12.5 m (the
    aperture reaches pad CMPs per side), h 0..2400 m, 4 ms; planes and diffractors, SNR 2."""
    fold, ns = PAPER_SHAPES[shape]
    rng = np.random.default_rng(seed + 1000)
    ds = crs_line(n_central + 2 * pad, fold, ns, 0.004, 0.0, 2400.0,
                  int(rng.integers(3, 5)), int(rng.integers(2, 4)), 2.0, seed)
    ds["central"] = np.arange(pad, pad + n_central, dtype=np.int32)
    ds["apm"] = pad * 12.5
    return ds


def crs_ranges(max_dip_deg=20.0, vmin=1500.0, vlo=1400.0, vhi=4500.0):
    """(lo, hi) of A, B, C for the CRS grids: A = +-2 sin(dip)/vmin, B = +-4/vlo^2,
    C = 4/v^2 over [vlo, vhi]."""
    amax = 2.0 * np.sin(np.deg2rad(max_dip_deg)) / vmin
    cmax = 4.0 / vlo ** 2
    cmin = 4.0 / vhi ** 2
    return (-amax, amax), (-cmax, cmax), (cmin, cmax)


# --- batched uneven items --------------------------------------------------------------

# numpy mirror of the seis_batch_item layout (64 bytes; field order and types as in the C ABI)
BATCH_ITEM_DTYPE = np.dtype([("trace_begin", "<i8"), ("trace_end", "<i8"), ("out_begin", "<i8"),
                             ("rows", "<i4"), ("kind", "<i4"), ("dt", "<f4"), ("m_c", "<f4"),
                             ("a_off", "<i4"), ("nA", "<i4"), ("b_off", "<i4"), ("nB", "<i4"),
                             ("c_off", "<i4"), ("nC", "<i4")])


def score_cube(rows, ncand, levels=7, seed=9):
    """Seeded scores in [0, 1) on a few levels (so rows hold many ties), float32
    [rows, ncand]: input for the selection of refinement starts."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, levels, size=(rows, ncand)) / levels).astype(np.float32)


def batch_workload(n_items=10000, seed=4, fold=(8, 120), ns=(1000, 4000), dts=(0.002, 0.004),
                   nc_range=(101, 201), crs_grid=(11, 11, 21), p_crs=0.5, snr=2.0,
                   max_dm=125.0, hmax=2500.0):
    """Uneven items: each a CMP gather (prob 1 - p_crs) or a CRS supergather whose traces
    carry their own midpoint offsets dm ~ U(-max_dm, max_dm).  Fold ~ U{fold}, samples ~
    U{ns}, dt from dts.  CMP items search nc ~ U{nc_range} values of C = 4/v^2 (v in
    1400..4500 m/s); CRS items the crs_grid over crs_ranges().  Events: dipping planes
    through the item centre (exact CRS form) and, for CMP items, hyperbolae.  Items come out
    sorted by cost per 32-row task (fold x candidates), largest first.
    Returns (dataset dict, items structured array, poolA, poolB, poolC)."""
    rng = np.random.default_rng(seed)
    (alo, ahi), (blo, bhi), (clo, chi) = crs_ranges()
    poolA = np.linspace(alo, ahi, crs_grid[0]).astype(np.float32)
    poolB = np.linspace(blo, bhi, crs_grid[1]).astype(np.float32)
    cmp_grids = {nc: (4.0 / np.linspace(1400.0, 4500.0, nc) ** 2).astype(np.float32)
                 for nc in range(nc_range[0], nc_range[1] + 1)}
    pieces = [np.linspace(clo, chi, crs_grid[2]).astype(np.float32)]
    c_off_of = {}
    off = crs_grid[2]
    for nc, gvals in cmp_grids.items():
        c_off_of[nc] = off
        pieces.append(gvals)
        off += nc
    poolC = np.concatenate(pieces)
    kinds = (rng.random(n_items) < p_crs).astype(np.int32)
    folds = rng.integers(fold[0], fold[1] + 1, n_items)
    nss = rng.integers(ns[0], ns[1] + 1, n_items)
    dtv = np.asarray(dts, np.float64)[rng.integers(0, len(dts), n_items)]
    ncs = rng.integers(nc_range[0], nc_range[1] + 1, n_items)
    cost = folds * np.where(kinds == 1, int(np.prod(crs_grid)), ncs)
    order = np.argsort(-cost, kind="stable")
    kinds, folds, nss, dtv, ncs = kinds[order], folds[order], nss[order], dtv[order], ncs[order]
    trace_off = [0]
    traces, hs, ms = [], [], []
    items = np.zeros(n_items, BATCH_ITEM_DTYPE)
    tb = 0
    ob = 0
    for i in range(n_items):
        M, L, dt, kind = int(folds[i]), int(nss[i]), float(dtv[i]), int(kinds[i])
        T = L * dt
        mcen = 1000.0 * i
        h = rng.uniform(0.0, hmax, M)
        dm = rng.uniform(-max_dm, max_dm, M) if kind else np.zeros(M)
        blk = np.zeros((M, L))
        times, amps = [], []
        for _ in range(int(rng.integers(2, 5))):
            v = rng.uniform(1500.0, 4000.0)
            a = np.deg2rad(rng.uniform(-20.0, 20.0)) if kind else 0.0
            t0 = rng.uniform(0.2, 0.85 * T)
            p = t0 + 2.0 * np.sin(a) * dm / v
            t = np.where(p > 0, np.sqrt(np.maximum(p, 0) ** 2 + 4.0 * np.cos(a) ** 2 * h ** 2 / v ** 2),
                         np.nan)
            times.append(t)
            amps.append(np.full(M, rng.uniform(0.5, 1.0) * rng.choice([-1.0, 1.0])))
        _add_events_uniform(blk, np.array(times), np.array(amps), dt)
        if snr:
            sig = _noise_sigma(blk.reshape(1, -1), snr)[0]
            blk += np.random.default_rng([seed, 7, i]).standard_normal(blk.shape) * sig
        traces.append(blk.astype(np.float32).reshape(-1))
        trace_off.extend(list(trace_off[-1] + L * np.arange(1, M + 1)))
        hs.append(h.astype(np.float32))
        ms.append((mcen + dm).astype(np.float32))
        it = items[i]
        it["trace_begin"], it["trace_end"] = tb, tb + M
        it["out_begin"], it["rows"], it["kind"] = ob, L, kind
        it["dt"], it["m_c"] = dt, mcen
        if kind:
            it["a_off"], it["nA"], it["b_off"], it["nB"] = 0, crs_grid[0], 0, crs_grid[1]
            it["c_off"], it["nC"] = 0, crs_grid[2]
        else:
            it["a_off"], it["nA"], it["b_off"], it["nB"] = 0, 1, 0, 1
            it["c_off"], it["nC"] = c_off_of[int(ncs[i])], int(ncs[i])
        tb += M
        ob += L
    ntr = tb
    ds = dict(traces=np.concatenate(traces), trace_off=np.asarray(trace_off, np.int64),
              h=np.concatenate(hs), m=np.concatenate(ms),
              gather_off=np.array([0, ntr], np.int64), out_off=np.array([0, ob], np.int64),
              dt=np.float32([dtv[0]]), out_rows=ob)
    return ds, items, poolA, poolB, poolC
