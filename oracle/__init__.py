"""FP64 CPU oracle of the CMP / CRS semblance search (arXiv:1907.11678).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path (the CUDA library and
its Python binding) never does.  The arithmetic lives in ``seis_oracle.c`` (plain C,
FP64, OpenMP over output rows); this module compiles it with gcc and marshals numpy
arrays into it.  It shares no code with the CUDA implementation.

Pins (tests/test_oracle.py): closed forms and invariants of Eq. 1 (constant traces,
a single trace, zero data, Cauchy-Schwarz bounds), an exactly-sampled hyperbolic
event and an exactly-sampled dipping plane (S = 1 at the true operator), a
hand-derived worked example under tests/golden/, a pure-Python brute force on tiny
inputs, numpy.interp for the stack of a single trace, the CRS -> CMP reductions and
central finite differences of the gradient.  The refinement (reading c16): its BFGS
update by the secant condition, symmetry, positive definiteness, the direct (Hessian)
form of the same update and the quadratic-termination property; its trajectory by a
hand-worked two-step case (with the C axis alone active, the second step is the secant
step of one-dimensional BFGS) and by its invariants (monotone S, bounds respected, the
exact operator of a sampled plane reached from a nearby start, the best of several
starts never below any one of them).  The start selection (top_starts) is pinned by
hand-worked rows with ties.  The admissible ranges of S, stack and N where FP32 rounding
may decide a trace's participation either way (reading c5) are pinned by brute force
over the flagged traces in and out.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seis_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libseis_oracle.so")
_lib = None
_lock = threading.Lock()

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp); returns the shared-library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.seis_oracle_cmp.restype = ctypes.c_int
            lib.seis_oracle_cmp_t0win.restype = ctypes.c_int
            lib.seis_oracle_crs.restype = ctypes.c_int
            lib.seis_oracle_crs_t0win.restype = ctypes.c_int
            lib.seis_oracle_crs_eval.restype = ctypes.c_int
            lib.seis_oracle_crs_refine.restype = ctypes.c_int
            lib.seis_oracle_neighbours.restype = ctypes.c_int
            lib.seis_oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def max_threads() -> int:
    return int(_load().seis_oracle_max_threads())


def velocity_grid(vmin: float, vmax: float, nc: int) -> np.ndarray:
    """Section 3.2: nc velocities linearly spaced in [vmin, vmax]; returns C = 4/v^2 (FP64)."""
    out = np.empty(nc, np.float64)
    _load().seis_oracle_velocity_grid(ctypes.c_double(vmin), ctypes.c_double(vmax),
                                      ctypes.c_int32(nc), _p(out))
    return out


def linear_grid(lo: float, hi: float, n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().seis_oracle_linear_grid(ctypes.c_double(lo), ctypes.c_double(hi),
                                    ctypes.c_int32(n), _p(out))
    return out


class Result(dict):
    """Attribute access to the oracle's output arrays."""
    __getattr__ = dict.__getitem__


class _Ranges(ctypes.Structure):
    """oracle_ranges of seis_oracle.c: per entry, the admissible range of S, the stack and N
    over the outcomes FP32 rounding may give the flagged traces (reading c5), and the stack
    at the entry."""
    _fields_ = [("S_lo", _vp), ("S_hi", _vp), ("stack", _vp), ("st_lo", _vp), ("st_hi", _vp),
                ("N_lo", _vp), ("N_hi", _vp)]


def _ranges(shape):
    """Output arrays of the admissible ranges and the ctypes structure pointing at them."""
    arr = dict(S_lo=np.empty(shape, np.float64), S_hi=np.empty(shape, np.float64),
               stack_at=np.empty(shape, np.float64), st_lo=np.empty(shape, np.float64),
               st_hi=np.empty(shape, np.float64), N_lo=np.empty(shape, np.int32),
               N_hi=np.empty(shape, np.int32))
    st = _Ranges(_p(arr["S_lo"]), _p(arr["S_hi"]), _p(arr["stack_at"]), _p(arr["st_lo"]),
                 _p(arr["st_hi"]), _p(arr["N_lo"]), _p(arr["N_hi"]))
    return arr, st


def cmp_semblance(ds, C, w=11, rows=None, want_cube=True, knot_eps=1e-3, nthreads=0,
                  t0_window=False) -> Result:
    """CMP search (Eq. 1, Algorithm 1, Section 3.2) on dataset ``ds`` (dict of arrays:
    traces, trace_off, h, gather_off, out_off, dt).  ``rows``: global output rows to
    evaluate (default all).  Returns S [nrows, nc], N, edge, best_idx, best_S,
    second_S, stack (FP64 / int).  t0_window: the window over neighbouring output times
    instead (reading c18, seis_oracle_cmp_t0win)."""
    lib = _load()
    traces = _c(ds["traces"], np.float32)
    trace_off = _c(ds["trace_off"], np.int64)
    h = _c(ds["h"], np.float32)
    gather_off = _c(ds["gather_off"], np.int64)
    out_off = _c(ds["out_off"], np.int64)
    dt = _c(ds["dt"], np.float32)
    C = _c(C, np.float32)
    G = len(gather_off) - 1
    nc = len(C)
    rows_a = None if rows is None else _c(rows, np.int64)
    nrows = int(out_off[-1]) if rows is None else len(rows_a)
    S = np.empty((nrows, nc), np.float64) if want_cube else None
    N = np.empty((nrows, nc), np.int32) if want_cube else None
    edge = np.empty((nrows, nc), np.int8) if want_cube else None
    rng, rst = _ranges((nrows, nc)) if want_cube else ({}, None)
    bi = np.empty(nrows, np.int32)
    bs = np.empty(nrows, np.float64)
    b2 = np.empty(nrows, np.float64)
    st = np.empty(nrows, np.float64)
    fn = lib.seis_oracle_cmp_t0win if t0_window else lib.seis_oracle_cmp
    rc = fn(_p(traces), _p(trace_off), _p(h), _p(gather_off), _p(out_off),
            _p(dt), ctypes.c_int64(G), _p(C), ctypes.c_int32(nc),
            ctypes.c_int32(w), _p(rows_a), ctypes.c_int64(nrows),
            _p(S), _p(N), _p(edge), _p(bi), _p(bs), _p(b2), _p(st),
            ctypes.c_double(knot_eps), ctypes.c_int32(nthreads),
            None if rst is None else ctypes.byref(rst))
    if rc != 0:
        raise ValueError("seis_oracle_cmp: invalid arguments")
    return Result(S=S, N=N, edge=edge, best_idx=bi, best_S=bs, second_S=b2, stack=st, **rng)


def neighbours(ds, central, apm):
    """CRS aperture (Section 2.2, Section 3.5): traces whose midpoint lies within apm of
    the central gather's midpoint.  Returns (nbr_off int64 [n+1], nbr_trace int32, m_c f32)."""
    lib = _load()
    m = _c(ds["m"], np.float32)
    gather_off = _c(ds["gather_off"], np.int64)
    central = _c(central, np.int32)
    G = len(gather_off) - 1
    n = len(central)
    off = np.empty(n + 1, np.int64)
    mc = np.empty(n, np.float32)
    rc = lib.seis_oracle_neighbours(_p(m), _p(gather_off), ctypes.c_int64(G), _p(central),
                                    ctypes.c_int64(n), ctypes.c_double(apm), _p(off), None, _p(mc))
    if rc != 0:
        raise ValueError("seis_oracle_neighbours: invalid arguments")
    tr = np.empty(int(off[-1]), np.int32)
    lib.seis_oracle_neighbours(_p(m), _p(gather_off), ctypes.c_int64(G), _p(central),
                               ctypes.c_int64(n), ctypes.c_double(apm), _p(off), _p(tr), _p(mc))
    return off, tr, mc


def aperture(ds, central, apm):
    """The full neighbour description the CRS functions take: (nbr_off, nbr_trace, m_c,
    out_off_c, dt_c), where the output rows of central i are those of its own gather."""
    off, tr, mc = neighbours(ds, central, apm)
    central = np.asarray(central, np.int64)
    out_off = np.asarray(ds["out_off"], np.int64)
    ns = out_off[central + 1] - out_off[central]
    out_off_c = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    return off, tr, mc, out_off_c, np.asarray(ds["dt"], np.float32)[central]


def _crs_common(ds, nb):
    off, tr, mc, out_off_c, dt_c = nb
    return (_c(ds["traces"], np.float32), _c(ds["trace_off"], np.int64), _c(ds["h"], np.float32),
            _c(ds["m"], np.float32), _c(off, np.int64), _c(tr, np.int32), _c(mc, np.float32),
            _c(out_off_c, np.int64), _c(dt_c, np.float32))


def crs_semblance(ds, nb, A, B, C, w=11, rows=None, want_cube=False, knot_eps=1e-3,
                  nthreads=0, t0_window=False) -> Result:
    """CRS search over the flattened grid cand = (ia*nB + ib)*nC + ic.  ``nb`` =
    (nbr_off, nbr_trace, m_c, out_off_c, dt_c) describes the central CDPs.  t0_window: the
    window over neighbouring output times (reading c18, seis_oracle_crs_t0win)."""
    lib = _load()
    arrs = _crs_common(ds, nb)
    A = _c(A, np.float32); B = _c(B, np.float32); C = _c(C, np.float32)
    ncen = len(arrs[6])
    ncand = len(A) * len(B) * len(C)
    rows_a = None if rows is None else _c(rows, np.int64)
    nrows = int(arrs[7][-1]) if rows is None else len(rows_a)
    S = np.empty((nrows, ncand), np.float64) if want_cube else None
    N = np.empty((nrows, ncand), np.int32) if want_cube else None
    edge = np.empty((nrows, ncand), np.int8) if want_cube else None
    rng, rst = _ranges((nrows, ncand)) if want_cube else ({}, None)
    bi = np.empty(nrows, np.int32)
    bs = np.empty(nrows, np.float64)
    b2 = np.empty(nrows, np.float64)
    st = np.empty(nrows, np.float64)
    fn = lib.seis_oracle_crs_t0win if t0_window else lib.seis_oracle_crs
    rc = fn(*[_p(a) for a in arrs], ctypes.c_int64(ncen),
            _p(A), ctypes.c_int32(len(A)), _p(B), ctypes.c_int32(len(B)),
            _p(C), ctypes.c_int32(len(C)), ctypes.c_int32(w),
            _p(rows_a), ctypes.c_int64(nrows),
            _p(S), _p(N), _p(edge), _p(bi), _p(bs), _p(b2), _p(st),
            ctypes.c_double(knot_eps), ctypes.c_int32(nthreads),
            None if rst is None else ctypes.byref(rst))
    if rc != 0:
        raise ValueError("seis_oracle_crs: invalid arguments")
    return Result(S=S, N=N, edge=edge, best_idx=bi, best_S=bs, second_S=b2, stack=st, **rng)


def crs_eval(ds, nb, theta, w=11, rows=None, knot_eps=1e-4, nthreads=0) -> Result:
    """S, dS/d(A,B,C) and stack at one operator per row (theta [nrows, 3]).  ``knot`` flags
    rows where a trace lies within knot_eps*(1 + 3e-3 u) samples of a sample point or a
    mask edge (the gradient is defined almost everywhere; FP32 may land on either side)."""
    lib = _load()
    arrs = _crs_common(ds, nb)
    ncen = len(arrs[6])
    rows_a = None if rows is None else _c(rows, np.int64)
    nrows = int(arrs[7][-1]) if rows is None else len(rows_a)
    theta = _c(theta, np.float64).reshape(nrows, 3)
    S = np.empty(nrows, np.float64)
    grad = np.empty((nrows, 3), np.float64)
    st = np.empty(nrows, np.float64)
    N = np.empty(nrows, np.int32)
    knot = np.empty(nrows, np.int8)
    rng, rst = _ranges(nrows)
    rc = lib.seis_oracle_crs_eval(*[_p(a) for a in arrs], ctypes.c_int64(ncen), ctypes.c_int32(w),
                                  _p(rows_a), ctypes.c_int64(nrows), _p(theta),
                                  _p(S), _p(grad), _p(st), _p(N), _p(knot),
                                  ctypes.c_double(knot_eps), ctypes.c_int32(nthreads),
                                  ctypes.byref(rst))
    if rc != 0:
        raise ValueError("seis_oracle_crs_eval: invalid arguments")
    rng.pop("stack_at")
    return Result(S=S, grad=grad, stack=st, N=N, knot=knot != 0, **rng)


def crs_refine(ds, nb, theta0, lo3, hi3, steps=20, step0=0.05, w=11, rows=None,
               nthreads=0) -> Result:
    """Projected quasi-Newton (BFGS) gradient ascent from theta0 in normalised coordinates,
    with step halving on rejected trials (reading c16).  Returns theta, S, grad, stack and
    traj [nrows, steps, 5]: each trial's operator (A, B, C), its S and whether it was
    accepted (NaN for trials never made)."""
    lib = _load()
    arrs = _crs_common(ds, nb)
    ncen = len(arrs[6])
    rows_a = None if rows is None else _c(rows, np.int64)
    nrows = int(arrs[7][-1]) if rows is None else len(rows_a)
    theta0 = _c(theta0, np.float64).reshape(nrows, 3)
    lo3 = _c(lo3, np.float64); hi3 = _c(hi3, np.float64)
    th = np.empty((nrows, 3), np.float64)
    S = np.empty(nrows, np.float64)
    grad = np.empty((nrows, 3), np.float64)
    st = np.empty(nrows, np.float64)
    traj = np.empty((nrows, max(steps, 0), 5), np.float64)
    rc = lib.seis_oracle_crs_refine(*[_p(a) for a in arrs], ctypes.c_int64(ncen),
                                    ctypes.c_int32(w), _p(rows_a), ctypes.c_int64(nrows),
                                    _p(theta0), _p(lo3), _p(hi3), ctypes.c_int32(steps),
                                    ctypes.c_double(step0), _p(th), _p(S), _p(grad), _p(st),
                                    ctypes.c_int32(nthreads), _p(traj))
    if rc != 0:
        raise ValueError("seis_oracle_crs_refine: invalid arguments")
    return Result(theta=th, S=S, grad=grad, stack=st, traj=traj)


def bfgs_inverse_update(H, s, y):
    """The refinement's BFGS update of a 3x3 inverse curvature estimate H with step s and
    gradient change y (returns the updated copy)."""
    H9 = _c(np.array(H, np.float64).reshape(9), np.float64).copy()
    _load().seis_oracle_bfgs_inverse_update(_p(H9), _p(_c(s, np.float64)), _p(_c(y, np.float64)))
    return H9.reshape(3, 3)


def top_starts(S_cube, A, B, C, nstart):
    """The nstart best candidates of every row of a CRS cube [rows, nA*nB*nC], ordered by
    S descending and candidate index ascending on ties, as operators [nstart, rows, 3]
    with cand = (ia*nB + ib)*nC + ic (the starts of a multi-start refinement, reading c16).
    Plain definition: a stable sort of each row."""
    S_cube = np.asarray(S_cube)
    A, B, C = (np.asarray(v) for v in (A, B, C))
    nB, nC = len(B), len(C)
    out = np.empty((nstart, S_cube.shape[0], 3), np.float64)
    for r in range(S_cube.shape[0]):
        order = sorted(range(S_cube.shape[1]), key=lambda c: (-S_cube[r, c], c))[:nstart]
        for j, c in enumerate(order):
            out[j, r] = (A[c // (nB * nC)], B[(c // nC) % nB], C[c % nC])
    return out


def local_max_flags(S_cube, nA, nB, nC):
    """Local maxima of each row's cube over the grid [nA, nB, nC]: entry c is one when its
    (S, -c) exceeds that of every neighbour (ia, ib, ic each within +-1, inside the grid).
    Plain definition, vectorised over rows: returns bool [rows, nA*nB*nC]."""
    S = np.asarray(S_cube, np.float64).reshape(-1, nA, nB, nC)
    idx = np.arange(nA * nB * nC).reshape(nA, nB, nC)
    is_max = np.ones(S.shape, bool)
    for da in (-1, 0, 1):
        for db in (-1, 0, 1):
            for dc in (-1, 0, 1):
                if da == db == dc == 0:
                    continue
                # target slice [a0:a1] sees neighbours at [a0+da : a1+da]
                sa = slice(max(0, -da), nA - max(0, da)); na = slice(max(0, da), nA + min(0, da))
                sb = slice(max(0, -db), nB - max(0, db)); nbs = slice(max(0, db), nB + min(0, db))
                sc = slice(max(0, -dc), nC - max(0, dc)); ncs = slice(max(0, dc), nC + min(0, dc))
                v, u = S[:, sa, sb, sc], S[:, na, nbs, ncs]
                iv, iu = idx[sa, sb, sc], idx[na, nbs, ncs]
                beaten = (u > v) | ((u == v) & (iu < iv))
                is_max[:, sa, sb, sc] &= ~beaten
    return is_max.reshape(S.shape[0], -1)


def local_max_starts(S_cube, A, B, C, nstart):
    """Starts at the cube's local maxima: per row, the local maxima (local_max_flags) in the
    order S descending, candidate index ascending, then the other candidates in that order;
    the first nstart, decoded to operators [nstart, rows, 3] (cand = (ia*nB + ib)*nC + ic)."""
    S_cube = np.asarray(S_cube, np.float64)
    A, B, C = (np.asarray(v) for v in (A, B, C))
    nA, nB, nC = len(A), len(B), len(C)
    flags = local_max_flags(S_cube, nA, nB, nC)
    idx = np.broadcast_to(np.arange(S_cube.shape[1]), S_cube.shape)
    order = np.lexsort((idx, -S_cube, ~flags), axis=-1)[:, :nstart]      # last key first
    ia, rem = np.divmod(order, nB * nC)
    ib, ic = np.divmod(rem, nC)
    return np.stack([A[ia], B[ib], C[ic]], axis=-1).transpose(1, 0, 2).astype(np.float64)


def crs_refine_multi(ds, nb, starts, lo3, hi3, steps=20, step0=0.05, w=11, rows=None,
                     nthreads=0) -> Result:
    """crs_refine from each start [nstart, rows, 3]; per row the result with the highest
    S is kept, the earlier start on ties (reading c16)."""
    best = None
    for k in range(len(starts)):
        r = crs_refine(ds, nb, starts[k], lo3, hi3, steps=steps, step0=step0, w=w, rows=rows,
                       nthreads=nthreads)
        r.pop("traj")
        if best is None:
            best = r
            continue
        better = r.S > best.S
        for key in ("theta", "S", "grad", "stack"):
            best[key][better] = r[key][better]
    return best


def offset_limited(ds, nb, hmax):
    """The neighbour description nb restricted to traces with |h| <= hmax (plain filter of
    each central's list, order kept)."""
    off, tr, mc, out_off_c, dt_c = nb
    h = np.asarray(ds["h"], np.float32)
    new_off, new_tr = [0], []
    for c in range(len(off) - 1):
        t = np.asarray(tr[off[c]:off[c + 1]])
        keep = t[np.abs(h[t]) <= np.float32(hmax)]
        new_tr.append(keep)
        new_off.append(new_off[-1] + len(keep))
    tr2 = np.concatenate(new_tr).astype(np.int32) if new_tr else np.zeros(0, np.int32)
    return np.asarray(new_off, np.int64), tr2, mc, out_off_c, dt_c


def crs_pragmatic(ds, central, apm, hzo, A, B, C, c_zo, w=11, nthreads=0) -> Result:
    """CRS operator by two small searches (not in the paper): C from the central CMP's own
    traces (dm = 0, A = B = 0: the CMP traveltime of Section 2.1), then A, B from the
    aperture's traces with |h| <= hzo at C = c_zo, then S and stack of the combined
    operator over the full aperture (Eq. 1, Algorithm 1).  Also returns each search's
    best / second-best S for the pick-parity waiver."""
    A = np.asarray(A); B = np.asarray(B); C = np.asarray(C)
    nb_full = aperture(ds, central, apm)
    nb_cmp = aperture(ds, central, 0.0)
    nb_zo = offset_limited(ds, nb_full, hzo)
    r1 = crs_semblance(ds, nb_cmp, [0.0], [0.0], C, w=w, want_cube=True, nthreads=nthreads)
    r2 = crs_semblance(ds, nb_zo, A, B, [c_zo], w=w, want_cube=True, nthreads=nthreads)
    theta = np.stack([A[r2.best_idx // len(B)], B[r2.best_idx % len(B)],
                      C[r1.best_idx]], 1).astype(np.float64)
    e = crs_eval(ds, nb_full, theta, w=w, nthreads=nthreads)
    return Result(theta=theta, S=e.S, stack=e.stack, N=e.N, knot=e.knot,
                  gap_cmp=r1.best_S - r1.second_S, gap_zo=r2.best_S - r2.second_S,
                  edge_cmp=(r1.edge != 0).any(axis=1), edge_zo=(r2.edge != 0).any(axis=1))


def cmp_as_crs(ds, gathers=None):
    """Neighbour description that makes each gather its own CRS 'aperture' (dm = 0
    when all traces of a gather share one midpoint); used by the reduction tests."""
    gather_off = np.asarray(ds["gather_off"], np.int64)
    G = len(gather_off) - 1
    gathers = np.arange(G) if gathers is None else np.asarray(gathers)
    off = [0]
    tr = []
    for g in gathers:
        ids = np.arange(gather_off[g], gather_off[g + 1], dtype=np.int32)
        tr.append(ids)
        off.append(off[-1] + len(ids))
    m = np.asarray(ds["m"], np.float32)
    mc = np.array([m[gather_off[g]] for g in gathers], np.float32)
    out_off = np.asarray(ds["out_off"], np.int64)
    ns = np.array([out_off[g + 1] - out_off[g] for g in gathers], np.int64)
    out_off_c = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    dt_c = np.asarray(ds["dt"], np.float32)[gathers]
    return (np.array(off, np.int64), np.concatenate(tr) if tr else np.zeros(0, np.int32),
            mc, out_off_c, dt_c)
