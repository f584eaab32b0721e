"""Thin Python binding of libseis (include/seis.h): argument marshalling only.

Device memory and streams come from PyTorch; every step of the semblance search runs
in the library's CUDA kernels.  If libseis.so is missing or no GPU is present the calls
raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass, field

import numpy as np
import torch

from . import build as _build

SEIS_OK, SEIS_EINVAL, SEIS_ECUDA, SEIS_ETIMEOUT, SEIS_EUNSUPPORTED = 0, -1, -2, -3, -4
SEIS_MAX_TRACE_SAMPLES = 12280
SEIS_MAX_W = 15

_lib = None
_lock = threading.Lock()


class SeisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libseis error {code}: {msg}")
        self.code = code


class _Gathers(ctypes.Structure):
    _fields_ = [("traces", ctypes.c_void_p), ("trace_off", ctypes.c_void_p),
                ("half_offset", ctypes.c_void_p), ("midpoint", ctypes.c_void_p),
                ("gather_off", ctypes.c_void_p), ("out_off", ctypes.c_void_p),
                ("dt", ctypes.c_void_p), ("ngathers", ctypes.c_int64),
                ("ntraces", ctypes.c_int64), ("max_rows", ctypes.c_int32),
                ("max_trace_samples", ctypes.c_int32)]


class _Aperture(ctypes.Structure):
    _fields_ = [("nbr_off", ctypes.c_void_p), ("nbr_trace", ctypes.c_void_p),
                ("m_c", ctypes.c_void_p), ("out_off", ctypes.c_void_p),
                ("dt", ctypes.c_void_p), ("n_central", ctypes.c_int64),
                ("max_rows", ctypes.c_int32), ("pad_", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None):
    """Load libseis.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _build.LIB
            if not os.path.exists(p):
                raise RuntimeError(f"libseis.so not found at {p}: run "
                                   "paper_1907_11678_gb300.build.build() first")
            lib = ctypes.CDLL(p)
            vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
            lib.seis_last_error.restype = ctypes.c_char_p
            lib.seis_device_status.argtypes = [vp]
            lib.cmp_semblance.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp]
            lib.cmp_semblance_t0win.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp]
            lib.crs_semblance.argtypes = [vp, vp, vp, i32, vp, i32, vp, i32, i32,
                                          vp, vp, vp, vp, vp, vp]
            lib.crs_semblance_t0win.argtypes = lib.crs_semblance.argtypes
            lib.seis_search_workspace_size.argtypes = [i64, i32, i64, i64]
            lib.seis_search_workspace_size.restype = ctypes.c_size_t
            lib.cmp_semblance_ws.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp, vp,
                                             ctypes.c_size_t, i64, vp]
            lib.crs_semblance_ws.argtypes = [vp, vp, vp, i32, vp, i32, vp, i32, i32,
                                             vp, vp, vp, vp, vp, vp, ctypes.c_size_t, i64, vp]
            lib.seis_crs_aperture.argtypes = [vp, vp, i64, f32, vp, vp, i64, vp, vp, vp,
                                              vp, vp, vp, vp]
            lib.seis_search_variant_name.restype = ctypes.c_char_p
            lib.seis_search_variant_name.argtypes = [ctypes.c_int]
            lib.seis_set_search_variant.argtypes = [ctypes.c_int]
            lib.seis_autotune_cmp.argtypes = [vp, vp, i32, i32, vp, vp, vp, i32, vp, vp, vp]
            lib.seis_autotune_crs.argtypes = [vp, vp, vp, i32, vp, i32, vp, i32, i32, vp, vp, vp,
                                              i32, vp, vp, vp]
            lib.stack.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
            lib.crs_semblance_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
            lib.seis_refine_workspace_size.argtypes = [i64]
            lib.seis_refine_workspace_size.restype = ctypes.c_size_t
            lib.crs_refine.argtypes = [vp, vp, vp, vp, vp, i32, f32, i32, vp, vp, vp, vp,
                                       ctypes.c_size_t, i64, vp]
            lib.crs_top_starts.argtypes = [vp, i64, vp, i32, vp, i32, vp, i32, i32, vp, vp]
            lib.crs_local_max_starts.argtypes = lib.crs_top_starts.argtypes
            lib.seis_refine_multi_workspace_size.argtypes = [i64]
            lib.seis_refine_multi_workspace_size.restype = ctypes.c_size_t
            lib.crs_refine_multi.argtypes = [vp, vp, vp, i32, vp, vp, i32, f32, i32, vp, vp, vp,
                                             vp, vp, ctypes.c_size_t, i64, vp]
            lib.seis_crs_aperture_offset.argtypes = [vp, vp, i64, f32, f32, vp, vp, i64, vp, vp,
                                                     vp, vp, vp, vp, vp]
            lib.seis_pragmatic_workspace_size.argtypes = [i64]
            lib.seis_pragmatic_workspace_size.restype = ctypes.c_size_t
            lib.crs_pragmatic.argtypes = [vp, vp, vp, vp, vp, i32, vp, i32, vp, i32, f32, i32, vp,
                                          vp, vp, vp, ctypes.c_size_t, i64, vp]
            lib.seis_batch_workspace_size.argtypes = [i64]
            lib.seis_batch_workspace_size.restype = ctypes.c_size_t
            lib.seis_batch_semblance.argtypes = [vp, vp, i64, vp, i32, vp, i32, vp, i32, i32, i32,
                                                 vp, vp, vp, vp, i64, vp, ctypes.c_size_t, vp]
            lib.seis_selftest_wait_timeout.argtypes = [i32, vp]
            lib.seis_velocity_grid.argtypes = [ctypes.c_double, ctypes.c_double, i32, vp, vp]
            lib.seis_selftest_fast_math.argtypes = [vp, vp]
            lib.seis_linear_grid.argtypes = [ctypes.c_double, ctypes.c_double, i32, vp, vp]
            lib.seis_autotune_batch.argtypes = [vp, vp, i64, vp, i32, vp, i32, vp, i32, i32, vp,
                                                vp, vp, vp, i64, vp, ctypes.c_size_t, i32, vp,
                                                vp, vp]
            lib.seis_autotune_save.argtypes = [ctypes.c_char_p]
            lib.seis_autotune_load.argtypes = [ctypes.c_char_p]
            for name in ("seis_device_status", "cmp_semblance", "crs_semblance",
                         "seis_crs_aperture", "seis_search_variant_count",
                         "seis_set_search_variant", "seis_get_search_variant",
                         "seis_autotune_cmp", "seis_autotune_crs", "seis_autotune_save",
                         "seis_autotune_load", "seis_autotune_clear", "stack",
                         "crs_semblance_grad", "crs_refine", "crs_top_starts",
                         "crs_local_max_starts",
                         "crs_refine_multi", "seis_batch_semblance", "seis_autotune_batch",
                         "seis_crs_aperture_offset", "crs_pragmatic", "cmp_semblance_t0win",
                         "crs_semblance_t0win", "seis_velocity_grid", "seis_linear_grid",
                         "cmp_semblance_ws", "crs_semblance_ws",
                         "seis_selftest_fast_math",
                         "seis_selftest_wait_timeout"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def _check(rc):
    if rc != SEIS_OK:
        raise SeisError(rc, load_library().seis_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _input(t, name: str, dev, numel: int | None = None, dtype=torch.float32) -> torch.Tensor:
    """An input array as a contiguous `dtype` tensor on the gathers' device (no copy when it
    already is one).  The kernels read `numel` elements through the pointer, so a shorter
    array is refused here rather than read out of bounds on the GPU."""
    t = torch.as_tensor(t).to(device=dev, dtype=dtype).contiguous()
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, the call reads {numel}")
    return t


def _output(out: dict, key: str, dev, dtype, numel: int) -> torch.Tensor | None:
    """A caller-provided output tensor (or None when absent).  The kernels write it in
    place, so it must already be contiguous, of `dtype`, on the gathers' device and hold at
    least `numel` elements."""
    t = out.get(key)
    if t is None:
        return None
    if (not isinstance(t, torch.Tensor) or t.device != dev or t.dtype != dtype
            or not t.is_contiguous() or t.numel() < numel):
        raise ValueError(f"out[{key!r}] must be a contiguous {dtype} tensor on {dev} with at "
                         f"least {numel} elements")
    return t


def _rows_out(dev, rows: int, abc: bool) -> dict:
    """Fresh best_idx, best_C or best_ABC, best_S and stack outputs for `rows` rows."""
    out = dict(best_idx=torch.empty(rows, dtype=torch.int32, device=dev))
    if abc:
        out["best_ABC"] = torch.empty((rows, 3), dtype=torch.float32, device=dev)
    else:
        out["best_C"] = torch.empty(rows, dtype=torch.float32, device=dev)
    out["best_S"] = torch.empty(rows, dtype=torch.float32, device=dev)
    out["stack"] = torch.empty(rows, dtype=torch.float32, device=dev)
    return out


def _check_rows_out(out: dict, dev, rows: int, ncand: int, abc: bool) -> None:
    """Check a caller-provided output dict of a search (see _rows_out; S is [rows, ncand])."""
    for key in ("best_idx", "best_S", "stack"):
        if out.get(key) is None:
            raise ValueError(f"out[{key!r}] is required")
    _output(out, "best_idx", dev, torch.int32, rows)
    _output(out, "best_ABC" if abc else "best_C", dev, torch.float32, rows * (3 if abc else 1))
    _output(out, "best_S", dev, torch.float32, rows)
    _output(out, "stack", dev, torch.float32, rows)
    _output(out, "S", dev, torch.float32, rows * ncand)


@dataclass
class Gathers:
    """A set of gathers resident on the GPU (arrays as in include/seis.h)."""
    traces: torch.Tensor
    trace_off: torch.Tensor
    h: torch.Tensor
    m: torch.Tensor | None
    gather_off: torch.Tensor
    out_off: torch.Tensor
    dt: torch.Tensor
    ngathers: int
    ntraces: int
    max_rows: int
    max_trace_samples: int
    rows: int
    _desc: _Gathers | None = field(default=None, repr=False)

    def descriptor(self) -> _Gathers:
        if self._desc is None:
            self._desc = _Gathers(self.traces.data_ptr(), self.trace_off.data_ptr(),
                                  self.h.data_ptr(),
                                  None if self.m is None else self.m.data_ptr(),
                                  self.gather_off.data_ptr(), self.out_off.data_ptr(),
                                  self.dt.data_ptr(), self.ngathers, self.ntraces,
                                  self.max_rows, self.max_trace_samples)
        return self._desc


def _check_dataset(traces, trace_off, h, m, gather_off, out_off, dt) -> None:
    """The offset arrays are the kernels' only bounds (include/seis.h), so a dataset whose
    offsets do not index inside its own arrays is refused here, on the host."""
    def monotone(name, a, lo, hi):
        if len(a) < 1 or a[0] < lo or a[-1] > hi or np.any(np.diff(a) < 0):
            raise ValueError(f"{name} must be non-decreasing within [{lo}, {hi}]")
    ntr = len(trace_off) - 1
    G = len(gather_off) - 1
    monotone("trace_off", trace_off, 0, len(traces))
    monotone("gather_off", gather_off, 0, ntr)
    if len(out_off) != G + 1:
        raise ValueError(f"out_off needs {G + 1} entries (one per gather, plus one)")
    monotone("out_off", out_off, 0, np.iinfo(np.int64).max)
    if len(h) != ntr or (m is not None and len(m) != ntr):
        raise ValueError(f"h (and m) need one entry per trace ({ntr})")
    if len(dt) != G:
        raise ValueError(f"dt needs one entry per gather ({G})")


def to_device(ds: dict, device="cuda", non_blocking=False) -> Gathers:
    """Copy a dataset dict (numpy arrays, see synth.py) to the GPU, after checking that its
    offsets index inside its arrays."""
    def t(a, dt):
        x = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
        if non_blocking:
            x = x.pin_memory()
        return x.to(device, non_blocking=non_blocking)
    trace_off = np.asarray(ds["trace_off"], np.int64)
    out_off = np.asarray(ds["out_off"], np.int64)
    gather_off = np.asarray(ds["gather_off"], np.int64)
    _check_dataset(np.ravel(ds["traces"]), trace_off, np.ravel(ds["h"]),
                   None if ds.get("m") is None else np.ravel(ds["m"]), gather_off, out_off,
                   np.ravel(ds["dt"]))
    return Gathers(traces=t(ds["traces"], np.float32), trace_off=t(trace_off, np.int64),
                   h=t(ds["h"], np.float32),
                   m=t(ds["m"], np.float32) if ds.get("m") is not None else None,
                   gather_off=t(gather_off, np.int64), out_off=t(out_off, np.int64),
                   dt=t(ds["dt"], np.float32), ngathers=len(gather_off) - 1,
                   ntraces=len(trace_off) - 1,
                   max_rows=int(np.diff(out_off).max()),
                   max_trace_samples=int(np.diff(trace_off).max()) if len(trace_off) > 1 else 0,
                   rows=int(out_off[-1]))


def velocity_grid(vmin: float, vmax: float, nc: int, device="cuda", stream=None) -> torch.Tensor:
    """Candidate grid of Section 3.2, C = 4/v^2 for nc velocities linearly spaced over
    [vmin, vmax] (include/seis.h: seis_velocity_grid), as a device tensor."""
    lib = load_library()
    out = torch.empty(int(nc), dtype=torch.float32, device=device)
    _check(lib.seis_velocity_grid(ctypes.c_double(vmin), ctypes.c_double(vmax), int(nc),
                                  _ptr(out), _stream_handle(stream)))
    return out


def linear_grid(lo: float, hi: float, n: int, device="cuda", stream=None) -> torch.Tensor:
    """A linear CRS parameter axis of n values over [lo, hi] (include/seis.h:
    seis_linear_grid), as a device tensor."""
    lib = load_library()
    out = torch.empty(int(n), dtype=torch.float32, device=device)
    _check(lib.seis_linear_grid(ctypes.c_double(lo), ctypes.c_double(hi), int(n), _ptr(out),
                                _stream_handle(stream)))
    return out


def _split_workspace(lib, dev, n_owner: int, max_rows: int, rows: int, ncand: int):
    """The scratch a split search needs on this device (None when it needs none)."""
    n = lib.seis_search_workspace_size(n_owner, max_rows, rows, ncand)
    return None if n == 0 else torch.empty(n, dtype=torch.uint8, device=dev)


def cmp_semblance(g: Gathers, C: torch.Tensor, w: int = 11, want_cube: bool = False,
                  stream=None, out: dict | None = None, split: bool = False) -> dict:
    """CMP semblance search (include/seis.h: cmp_semblance).  Returns device tensors
    best_idx, best_C, best_S, stack (and S [rows, nc] when want_cube).  split: spread each
    tile's candidates over several CTAs when the gathers do not fill the GPU
    (cmp_semblance_ws; bit-identical results)."""
    lib = load_library()
    dev = g.traces.device
    C = _input(C, "C", dev)
    nc = int(C.numel())
    if out is None:
        out = _rows_out(dev, g.rows, abc=False)
        if want_cube:
            out["S"] = torch.empty((g.rows, nc), dtype=torch.float32, device=dev)
    else:
        _check_rows_out(out, dev, g.rows, nc, abc=False)
    if split:
        ws = _split_workspace(lib, dev, g.ngathers, g.max_rows, g.rows, nc)
        rc = lib.cmp_semblance_ws(ctypes.byref(g.descriptor()), _ptr(C), nc, w,
                                  _ptr(out.get("S")), _ptr(out["best_idx"]),
                                  _ptr(out.get("best_C")), _ptr(out["best_S"]), _ptr(out["stack"]),
                                  _ptr(ws), 0 if ws is None else ws.numel(), g.rows,
                                  _stream_handle(stream))
    else:
        rc = lib.cmp_semblance(ctypes.byref(g.descriptor()), _ptr(C), nc, w, _ptr(out.get("S")),
                               _ptr(out["best_idx"]), _ptr(out.get("best_C")),
                               _ptr(out["best_S"]), _ptr(out["stack"]), _stream_handle(stream))
    _check(rc)
    return out


def cmp_semblance_t0win(g: Gathers, C: torch.Tensor, w: int = 11, want_cube: bool = False,
                        stream=None, out: dict | None = None) -> dict:
    """CMP semblance with the window over neighbouring output times (include/seis.h:
    cmp_semblance_t0win).  Same outputs as cmp_semblance."""
    lib = load_library()
    dev = g.traces.device
    C = _input(C, "C", dev)
    nc = int(C.numel())
    if out is None:
        out = _rows_out(dev, g.rows, abc=False)
        if want_cube:
            out["S"] = torch.empty((g.rows, nc), dtype=torch.float32, device=dev)
    else:
        _check_rows_out(out, dev, g.rows, nc, abc=False)
    _check(lib.cmp_semblance_t0win(ctypes.byref(g.descriptor()), _ptr(C), nc, w,
                                   _ptr(out.get("S")), _ptr(out["best_idx"]),
                                   _ptr(out.get("best_C")), _ptr(out["best_S"]),
                                   _ptr(out["stack"]), _stream_handle(stream)))
    return out


@dataclass
class Aperture:
    nbr_off: torch.Tensor
    nbr_trace: torch.Tensor
    m_c: torch.Tensor
    out_off: torch.Tensor
    dt: torch.Tensor
    n_central: int
    max_rows: int
    rows: int
    _desc: _Aperture | None = field(default=None, repr=False)

    def descriptor(self) -> _Aperture:
        if self._desc is None:
            self._desc = _Aperture(self.nbr_off.data_ptr(), self.nbr_trace.data_ptr(),
                                   self.m_c.data_ptr(), self.out_off.data_ptr(),
                                   self.dt.data_ptr(), self.n_central, self.max_rows, 0)
        return self._desc


def crs_aperture(g: Gathers, central, apm: float, hmax: float | None = None,
                 stream=None) -> Aperture:
    """Build the CRS apertures of the central gathers (include/seis.h: seis_crs_aperture, or
    seis_crs_aperture_offset when hmax is given: only traces with |h| <= hmax)."""
    lib = load_library()
    dev = g.traces.device
    if isinstance(central, torch.Tensor):
        central = central.detach().cpu()
    central = torch.from_numpy(np.ascontiguousarray(np.asarray(central), np.int32)).to(dev)
    n = int(central.numel())
    nbr_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    m_c = torch.empty(n, dtype=torch.float32, device=dev)
    out_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    dt_c = torch.empty(n, dtype=torch.float32, device=dev)
    total = ctypes.c_int64(0)
    rows = ctypes.c_int64(0)
    mr = ctypes.c_int32(0)
    sh = _stream_handle(stream)
    args = (ctypes.byref(g.descriptor()), _ptr(central), n, ctypes.c_float(apm))
    if hmax is None:
        fn = lib.seis_crs_aperture
    else:
        fn = lib.seis_crs_aperture_offset
        args = args + (ctypes.c_float(hmax),)
    args = args + (_ptr(nbr_off),)
    _check(fn(*args, None, 0, _ptr(m_c), _ptr(out_off), _ptr(dt_c),
              ctypes.byref(total), ctypes.byref(rows), ctypes.byref(mr), sh))
    nbr_trace = torch.empty(max(1, total.value), dtype=torch.int32, device=dev)
    _check(fn(*args, _ptr(nbr_trace), total.value, _ptr(m_c), _ptr(out_off),
              _ptr(dt_c), None, None, None, sh))
    return Aperture(nbr_off, nbr_trace, m_c, out_off, dt_c, n, int(mr.value), int(rows.value))


def _crs_search(lib_fn, g, ap, A, B, C, w, want_cube, stream, out=None, split=False) -> dict:
    lib = load_library()
    dev = g.traces.device
    A, B, C = _input(A, "A", dev), _input(B, "B", dev), _input(C, "C", dev)
    nA, nB, nC = int(A.numel()), int(B.numel()), int(C.numel())
    if out is None:
        out = _rows_out(dev, ap.rows, abc=True)
        if want_cube:
            out["S"] = torch.empty((ap.rows, nA * nB * nC), dtype=torch.float32, device=dev)
    else:
        _check_rows_out(out, dev, ap.rows, nA * nB * nC, abc=True)
    args = (ctypes.byref(g.descriptor()), ctypes.byref(ap.descriptor()), _ptr(A), nA, _ptr(B),
            nB, _ptr(C), nC, w, _ptr(out.get("S")), _ptr(out["best_idx"]), _ptr(out["best_ABC"]),
            _ptr(out["best_S"]), _ptr(out["stack"]))
    if split:
        ws = _split_workspace(lib, dev, ap.n_central, ap.max_rows, ap.rows, nA * nB * nC)
        rc = lib.crs_semblance_ws(*args, _ptr(ws), 0 if ws is None else ws.numel(), ap.rows,
                                  _stream_handle(stream))
    else:
        rc = getattr(lib, lib_fn)(*args, _stream_handle(stream))
    _check(rc)
    return out


def crs_semblance(g: Gathers, ap: Aperture, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor,
                  w: int = 11, want_cube: bool = False, stream=None, out: dict | None = None,
                  split: bool = False) -> dict:
    """CRS semblance search over the flattened A x B x C grid (include/seis.h:
    crs_semblance).  Returns best_idx, best_ABC [rows, 3], best_S, stack (and S); `out`
    supplies the output tensors instead (as cmp_semblance); split as cmp_semblance
    (crs_semblance_ws)."""
    return _crs_search("crs_semblance", g, ap, A, B, C, w, want_cube, stream, out, split)


def crs_semblance_t0win(g: Gathers, ap: Aperture, A: torch.Tensor, B: torch.Tensor,
                        C: torch.Tensor, w: int = 11, want_cube: bool = False,
                        stream=None) -> dict:
    """CRS search with the window over neighbouring output times (include/seis.h:
    crs_semblance_t0win).  Same outputs as crs_semblance."""
    return _crs_search("crs_semblance_t0win", g, ap, A, B, C, w, want_cube, stream)


def search_variants() -> list[str]:
    """Names of the search kernel variants (index = variant id)."""
    lib = load_library()
    return [lib.seis_search_variant_name(i).decode() for i in range(lib.seis_search_variant_count())]


def set_search_variant(v: int) -> None:
    _check(load_library().seis_set_search_variant(int(v)))


def get_search_variant() -> int:
    return int(load_library().seis_get_search_variant())


def autotune_cmp(g: Gathers, C: torch.Tensor, w: int = 11, reps: int = 2, stream=None):
    """Time every search-kernel variant on this CMP problem (include/seis.h:
    seis_autotune_cmp); later calls in the same shape bucket use the fastest.  Returns
    (chosen variant, list of mean milliseconds per variant)."""
    lib = load_library()
    dev = g.traces.device
    C = _input(C, "C", dev)
    bi = torch.empty(g.rows, dtype=torch.int32, device=dev)
    bs = torch.empty(g.rows, dtype=torch.float32, device=dev)
    st = torch.empty(g.rows, dtype=torch.float32, device=dev)
    nv = lib.seis_search_variant_count()
    ms = (ctypes.c_float * nv)()
    chosen = ctypes.c_int32(-1)
    _check(lib.seis_autotune_cmp(ctypes.byref(g.descriptor()), _ptr(C), int(C.numel()), w,
                                 _ptr(bi), _ptr(bs), _ptr(st), reps, ctypes.byref(chosen), ms,
                                 _stream_handle(stream)))
    return int(chosen.value), list(ms)


def autotune_crs(g: Gathers, ap: "Aperture", A, B, C, w: int = 11, reps: int = 2, stream=None):
    """As autotune_cmp for a CRS problem (include/seis.h: seis_autotune_crs)."""
    lib = load_library()
    dev = g.traces.device
    A, B, C = _input(A, "A", dev), _input(B, "B", dev), _input(C, "C", dev)
    bi = torch.empty(ap.rows, dtype=torch.int32, device=dev)
    bs = torch.empty(ap.rows, dtype=torch.float32, device=dev)
    st = torch.empty(ap.rows, dtype=torch.float32, device=dev)
    nv = lib.seis_search_variant_count()
    ms = (ctypes.c_float * nv)()
    chosen = ctypes.c_int32(-1)
    _check(lib.seis_autotune_crs(ctypes.byref(g.descriptor()), ctypes.byref(ap.descriptor()),
                                 _ptr(A), int(A.numel()), _ptr(B), int(B.numel()), _ptr(C),
                                 int(C.numel()), w, _ptr(bi), _ptr(bs), _ptr(st), reps,
                                 ctypes.byref(chosen), ms, _stream_handle(stream)))
    return int(chosen.value), list(ms)


def autotune_save(path: str) -> None:
    _check(load_library().seis_autotune_save(path.encode()))


def autotune_load(path: str) -> None:
    _check(load_library().seis_autotune_load(path.encode()))


def autotune_clear() -> None:
    _check(load_library().seis_autotune_clear())


def stack(g: Gathers, ap: "Aperture | None", params: torch.Tensor, w: int = 11,
          stream=None) -> dict:
    """Stack (and semblance, trace count) along one operator per output row
    (include/seis.h: stack).  ap None: CMP, params [rows] = C; else CRS, params [rows, 3]."""
    lib = load_library()
    dev = g.traces.device
    rows = g.rows if ap is None else ap.rows
    params = _input(params, "params", dev, rows * (1 if ap is None else 3))
    out = dict(stack=torch.empty(rows, dtype=torch.float32, device=dev),
               S=torch.empty(rows, dtype=torch.float32, device=dev),
               N=torch.empty(rows, dtype=torch.int32, device=dev))
    _check(lib.stack(ctypes.byref(g.descriptor()),
                     None if ap is None else ctypes.byref(ap.descriptor()), _ptr(params), w,
                     _ptr(out["stack"]), _ptr(out["S"]), _ptr(out["N"]), _stream_handle(stream)))
    return out


def crs_semblance_grad(g: Gathers, ap: "Aperture", ABC: torch.Tensor, w: int = 11,
                       stream=None):
    """Semblance, dS/d(A,B,C) [rows, 3] and stack at ABC [rows, 3] (adjoint kernel)."""
    lib = load_library()
    dev = g.traces.device
    ABC = _input(ABC, "ABC", dev, ap.rows * 3)
    S = torch.empty(ap.rows, dtype=torch.float32, device=dev)
    grad = torch.empty((ap.rows, 3), dtype=torch.float32, device=dev)
    st = torch.empty(ap.rows, dtype=torch.float32, device=dev)
    _check(lib.crs_semblance_grad(ctypes.byref(g.descriptor()), ctypes.byref(ap.descriptor()),
                                  _ptr(ABC), w, _ptr(S), _ptr(grad), _ptr(st),
                                  _stream_handle(stream)))
    return S, grad, st


def crs_refine(g: Gathers, ap: "Aperture", ABC0: torch.Tensor, lo3, hi3, steps: int = 20,
               step0: float = 0.05, w: int = 11, stream=None, workspace=None) -> dict:
    """Gradient-ascent refinement of CRS operators from ABC0 [rows, 3] (include/seis.h:
    crs_refine).  Returns theta, S, grad, stack (device tensors)."""
    lib = load_library()
    dev = g.traces.device
    theta = _input(ABC0.detach(), "ABC0", dev, ap.rows * 3).clone()
    S = torch.empty(ap.rows, dtype=torch.float32, device=dev)
    grad = torch.empty((ap.rows, 3), dtype=torch.float32, device=dev)
    st = torch.empty(ap.rows, dtype=torch.float32, device=dev)
    nbytes = lib.seis_refine_workspace_size(ap.rows)
    if workspace is None or workspace.numel() < nbytes + 256:
        workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    lo = (ctypes.c_float * 3)(*[float(v) for v in lo3])
    hi = (ctypes.c_float * 3)(*[float(v) for v in hi3])
    _check(lib.crs_refine(ctypes.byref(g.descriptor()), ctypes.byref(ap.descriptor()),
                          _ptr(theta), lo, hi, int(steps), ctypes.c_float(step0), w, _ptr(S),
                          _ptr(grad), _ptr(st), ctypes.c_void_p(aligned),
                          workspace.numel() - (aligned - base), ap.rows, _stream_handle(stream)))
    return dict(theta=theta, S=S, grad=grad, stack=st)


def crs_top_starts(S_cube: torch.Tensor, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor,
                   nstart: int, stream=None, local_max: bool = False) -> torch.Tensor:
    """The nstart best coarse candidates of every row of a CRS cube [rows, nA*nB*nC] as
    operators [nstart, rows, 3] (include/seis.h: crs_top_starts; with local_max, the best
    local maxima of the cube first: crs_local_max_starts)."""
    lib = load_library()
    dev = S_cube.device
    A, B, C = _input(A, "A", dev), _input(B, "B", dev), _input(C, "C", dev)
    if S_cube.dim() != 2 or S_cube.shape[1] != A.numel() * B.numel() * C.numel():
        raise ValueError(f"S_cube must be [rows, {A.numel() * B.numel() * C.numel()}], "
                         f"got {tuple(S_cube.shape)}")
    S_cube = _input(S_cube, "S_cube", dev)
    rows = S_cube.shape[0]
    out = torch.empty((nstart, rows, 3), dtype=torch.float32, device=dev)
    fn = lib.crs_local_max_starts if local_max else lib.crs_top_starts
    _check(fn(_ptr(S_cube), rows, _ptr(A), A.numel(), _ptr(B), B.numel(), _ptr(C), C.numel(),
              int(nstart), _ptr(out), _stream_handle(stream)))
    return out


def crs_refine_multi(g: Gathers, ap: "Aperture", starts: torch.Tensor, lo3, hi3,
                     steps: int = 20, step0: float = 0.05, w: int = 11, stream=None,
                     workspace=None) -> dict:
    """crs_refine from each start [nstart, rows, 3], best S kept per row (include/seis.h:
    crs_refine_multi).  Returns theta, S, grad, stack (device tensors)."""
    lib = load_library()
    dev = g.traces.device
    if starts.dim() != 3 or starts.shape[1:] != (ap.rows, 3):
        raise ValueError(f"starts must be [nstart, {ap.rows}, 3], got {tuple(starts.shape)}")
    starts = _input(starts.detach(), "starts", dev)
    theta = torch.empty((ap.rows, 3), dtype=torch.float32, device=dev)
    S = torch.empty(ap.rows, dtype=torch.float32, device=dev)
    grad = torch.empty((ap.rows, 3), dtype=torch.float32, device=dev)
    st = torch.empty(ap.rows, dtype=torch.float32, device=dev)
    nbytes = lib.seis_refine_multi_workspace_size(ap.rows)
    if workspace is None or workspace.numel() < nbytes + 256:
        workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    lo = (ctypes.c_float * 3)(*[float(v) for v in lo3])
    hi = (ctypes.c_float * 3)(*[float(v) for v in hi3])
    _check(lib.crs_refine_multi(ctypes.byref(g.descriptor()), ctypes.byref(ap.descriptor()),
                                _ptr(starts), int(starts.shape[0]), lo, hi, int(steps),
                                ctypes.c_float(step0), w, _ptr(theta), _ptr(S), _ptr(grad),
                                _ptr(st), ctypes.c_void_p(aligned),
                                workspace.numel() - (aligned - base), ap.rows,
                                _stream_handle(stream)))
    return dict(theta=theta, S=S, grad=grad, stack=st)


def crs_pragmatic(g: Gathers, ap_full: "Aperture", ap_cmp: "Aperture", ap_zo: "Aperture",
                  A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, c_zo: float,
                  w: int = 11, stream=None, workspace=None) -> dict:
    """CRS operator from a central-CMP C search and a zero-offset (A, B) search, evaluated
    over the full aperture (include/seis.h: crs_pragmatic).  Returns theta, S, stack."""
    lib = load_library()
    dev = g.traces.device
    A, B, C = _input(A, "A", dev), _input(B, "B", dev), _input(C, "C", dev)
    theta = torch.empty((ap_full.rows, 3), dtype=torch.float32, device=dev)
    S = torch.empty(ap_full.rows, dtype=torch.float32, device=dev)
    st = torch.empty(ap_full.rows, dtype=torch.float32, device=dev)
    nbytes = lib.seis_pragmatic_workspace_size(ap_full.rows)
    if workspace is None or workspace.numel() < nbytes + 256:
        workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    _check(lib.crs_pragmatic(ctypes.byref(g.descriptor()), ctypes.byref(ap_full.descriptor()),
                             ctypes.byref(ap_cmp.descriptor()), ctypes.byref(ap_zo.descriptor()),
                             _ptr(A), A.numel(), _ptr(B), B.numel(), _ptr(C), C.numel(),
                             ctypes.c_float(c_zo), w, _ptr(theta), _ptr(S), _ptr(st),
                             ctypes.c_void_p(aligned), workspace.numel() - (aligned - base),
                             ap_full.rows, _stream_handle(stream)))
    return dict(theta=theta, S=S, stack=st)


class CRSSemblance(torch.autograd.Function):
    """S(A, B, C) per output row as a differentiable function of the operators [rows, 3]:
    forward runs the evaluation kernel, backward the hand-written adjoint kernel."""

    @staticmethod
    def forward(ctx, ABC, g, ap, w=11):
        out = stack(g, ap, ABC.detach().float(), w)
        ctx.save_for_backward(ABC.detach())
        ctx.g, ctx.ap, ctx.w = g, ap, w
        return out["S"]

    @staticmethod
    def backward(ctx, grad_S):
        (ABC,) = ctx.saved_tensors
        _, dS, _ = crs_semblance_grad(ctx.g, ctx.ap, ABC.float(), ctx.w)
        return grad_S.unsqueeze(1) * dS, None, None, None


def crs_semblance_at(ABC: torch.Tensor, g: Gathers, ap: "Aperture", w: int = 11):
    """Differentiable semblance of one CRS operator per row (see CRSSemblance)."""
    return CRSSemblance.apply(ABC, g, ap, w)


@dataclass
class Batch:
    """Batched items resident on the GPU (include/seis.h: seis_batch_item)."""
    items: torch.Tensor            # uint8 [nitems * 64], the raw item table
    nitems: int
    poolA: torch.Tensor
    poolB: torch.Tensor
    poolC: torch.Tensor
    out_rows: int
    workspace: torch.Tensor


def batch_to_device(items: np.ndarray, poolA, poolB, poolC, out_rows: int, device="cuda") -> Batch:
    """Copy a structured item array (synth.BATCH_ITEM_DTYPE) and the candidate pools."""
    lib = load_library()
    raw = torch.from_numpy(np.ascontiguousarray(items).view(np.uint8).copy()).to(device)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
    nbytes = lib.seis_batch_workspace_size(len(items))
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    return Batch(raw, len(items), f(poolA), f(poolB), f(poolC), int(out_rows), ws)


def batch_semblance(g: Gathers, b: Batch, w: int = 11, mode: int = 0, stream=None,
                    out: dict | None = None) -> dict:
    """Batched search over uneven CMP / CRS items (include/seis.h: seis_batch_semblance);
    mode 0 = one persistent launch, 1 = one launch per item."""
    lib = load_library()
    dev = g.traces.device
    if out is None:
        out = _rows_out(dev, b.out_rows, abc=True)
    else:
        _check_rows_out(out, dev, b.out_rows, 0, abc=True)
    base = b.workspace.data_ptr()
    aligned = (base + 255) & ~255
    _check(lib.seis_batch_semblance(
        ctypes.byref(g.descriptor()), _ptr(b.items), b.nitems, _ptr(b.poolA), int(b.poolA.numel()),
        _ptr(b.poolB), int(b.poolB.numel()), _ptr(b.poolC), int(b.poolC.numel()), w, mode,
        _ptr(out["best_idx"]), _ptr(out["best_ABC"]), _ptr(out["best_S"]), _ptr(out["stack"]),
        b.out_rows, ctypes.c_void_p(aligned), b.workspace.numel() - (aligned - base),
        _stream_handle(stream)))
    return out


def autotune_batch(g: Gathers, b: Batch, w: int = 11, reps: int = 1, stream=None):
    """Pick the batch kernel variant for window w by timing the persistent launch
    (include/seis.h: seis_autotune_batch).  Returns (chosen, ms per variant or -1)."""
    lib = load_library()
    dev = g.traces.device
    out = _rows_out(dev, b.out_rows, abc=True)
    base = b.workspace.data_ptr()
    aligned = (base + 255) & ~255
    nv = lib.seis_search_variant_count()
    ms = (ctypes.c_float * nv)()
    chosen = ctypes.c_int32(-1)
    _check(lib.seis_autotune_batch(
        ctypes.byref(g.descriptor()), _ptr(b.items), b.nitems, _ptr(b.poolA), int(b.poolA.numel()),
        _ptr(b.poolB), int(b.poolB.numel()), _ptr(b.poolC), int(b.poolC.numel()), w,
        _ptr(out["best_idx"]), _ptr(out["best_ABC"]), _ptr(out["best_S"]), _ptr(out["stack"]),
        b.out_rows, ctypes.c_void_p(aligned), b.workspace.numel() - (aligned - base), int(reps),
        ctypes.byref(chosen), ms, _stream_handle(stream)))
    return int(chosen.value), list(ms)


def selftest_wait_timeout(limit_us: int = 10000, stream=None) -> None:
    """Launch the bounded-wait self-test (include/seis.h: seis_selftest_wait_timeout)."""
    _check(load_library().seis_selftest_wait_timeout(int(limit_us), _stream_handle(stream)))


def selftest_fast_math(stream=None) -> tuple[float, float]:
    """Largest relative errors of the kernels' fast square root and reciprocal over every
    float in [1, 4) (include/seis.h: seis_selftest_fast_math)."""
    out = torch.empty(2, dtype=torch.float32, device="cuda")
    _check(load_library().seis_selftest_fast_math(_ptr(out), _stream_handle(stream)))
    e = out.cpu().tolist()
    return e[0], e[1]


def device_status(stream=None) -> None:
    """Raise if a kernel recorded a timed-out wait or an overflow since the last check."""
    _check(load_library().seis_device_status(_stream_handle(stream)))
