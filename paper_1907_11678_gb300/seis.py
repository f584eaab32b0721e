"""Thin Python binding of libseis (include/seis.h): argument marshalling only.

Device memory and streams come from PyTorch; every step of the semblance search runs
in the library's CUDA kernels.  If libseis.so is missing or no GPU is present the calls
raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
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
            lib.crs_semblance.argtypes = [vp, vp, vp, i32, vp, i32, vp, i32, i32,
                                          vp, vp, vp, vp, vp, vp]
            lib.seis_crs_aperture.argtypes = [vp, vp, i64, f32, vp, vp, i64, vp, vp, vp,
                                              vp, vp, vp, vp]
            lib.seis_search_variant_name.restype = ctypes.c_char_p
            lib.seis_search_variant_name.argtypes = [ctypes.c_int]
            lib.seis_set_search_variant.argtypes = [ctypes.c_int]
            for name in ("seis_device_status", "cmp_semblance", "crs_semblance",
                         "seis_crs_aperture", "seis_search_variant_count",
                         "seis_set_search_variant", "seis_get_search_variant"):
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


def to_device(ds: dict, device="cuda", non_blocking=False) -> Gathers:
    """Copy a dataset dict (numpy arrays, see synth.py) to the GPU."""
    def t(a, dt):
        x = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
        if non_blocking:
            x = x.pin_memory()
        return x.to(device, non_blocking=non_blocking)
    trace_off = np.asarray(ds["trace_off"], np.int64)
    out_off = np.asarray(ds["out_off"], np.int64)
    gather_off = np.asarray(ds["gather_off"], np.int64)
    return Gathers(traces=t(ds["traces"], np.float32), trace_off=t(trace_off, np.int64),
                   h=t(ds["h"], np.float32),
                   m=t(ds["m"], np.float32) if ds.get("m") is not None else None,
                   gather_off=t(gather_off, np.int64), out_off=t(out_off, np.int64),
                   dt=t(ds["dt"], np.float32), ngathers=len(gather_off) - 1,
                   ntraces=len(trace_off) - 1,
                   max_rows=int(np.diff(out_off).max()),
                   max_trace_samples=int(np.diff(trace_off).max()) if len(trace_off) > 1 else 0,
                   rows=int(out_off[-1]))


def velocity_grid(vmin: float, vmax: float, nc: int, device="cuda") -> torch.Tensor:
    """Candidate grid of Section 3.2: nc velocities linearly spaced in [vmin, vmax]
    (bounds included), as C = 4/v^2 in FP32."""
    v = np.linspace(vmin, vmax, nc, dtype=np.float64) if nc > 1 else np.array([vmin], np.float64)
    return torch.from_numpy((4.0 / v ** 2).astype(np.float32)).to(device)


def linear_grid(lo: float, hi: float, n: int, device="cuda") -> torch.Tensor:
    g = np.linspace(lo, hi, n, dtype=np.float64) if n > 1 else np.array([lo], np.float64)
    return torch.from_numpy(g.astype(np.float32)).to(device)


def cmp_semblance(g: Gathers, C: torch.Tensor, w: int = 11, want_cube: bool = False,
                  stream=None, out: dict | None = None) -> dict:
    """CMP semblance search (include/seis.h: cmp_semblance).  Returns device tensors
    best_idx, best_C, best_S, stack (and S [rows, nc] when want_cube)."""
    lib = load_library()
    dev = g.traces.device
    nc = int(C.numel())
    if out is None:
        out = dict(best_idx=torch.empty(g.rows, dtype=torch.int32, device=dev),
                   best_C=torch.empty(g.rows, dtype=torch.float32, device=dev),
                   best_S=torch.empty(g.rows, dtype=torch.float32, device=dev),
                   stack=torch.empty(g.rows, dtype=torch.float32, device=dev))
        if want_cube:
            out["S"] = torch.empty((g.rows, nc), dtype=torch.float32, device=dev)
    rc = lib.cmp_semblance(ctypes.byref(g.descriptor()), _ptr(C), nc, w, _ptr(out.get("S")),
                           _ptr(out["best_idx"]), _ptr(out.get("best_C")), _ptr(out["best_S"]),
                           _ptr(out["stack"]), _stream_handle(stream))
    _check(rc)
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


def crs_aperture(g: Gathers, central, apm: float, stream=None) -> Aperture:
    """Build the CRS apertures of the central gathers (include/seis.h: seis_crs_aperture)."""
    lib = load_library()
    dev = g.traces.device
    central = torch.as_tensor(np.asarray(central, np.int32)).to(dev)
    n = int(central.numel())
    nbr_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    m_c = torch.empty(n, dtype=torch.float32, device=dev)
    out_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    dt_c = torch.empty(n, dtype=torch.float32, device=dev)
    total = ctypes.c_int64(0)
    rows = ctypes.c_int64(0)
    mr = ctypes.c_int32(0)
    sh = _stream_handle(stream)
    args = (ctypes.byref(g.descriptor()), _ptr(central), n, ctypes.c_float(apm), _ptr(nbr_off))
    _check(lib.seis_crs_aperture(*args, None, 0, _ptr(m_c), _ptr(out_off), _ptr(dt_c),
                                 ctypes.byref(total), ctypes.byref(rows), ctypes.byref(mr), sh))
    nbr_trace = torch.empty(max(1, total.value), dtype=torch.int32, device=dev)
    _check(lib.seis_crs_aperture(*args, _ptr(nbr_trace), total.value, _ptr(m_c), _ptr(out_off),
                                 _ptr(dt_c), None, None, None, sh))
    return Aperture(nbr_off, nbr_trace, m_c, out_off, dt_c, n, int(mr.value), int(rows.value))


def crs_semblance(g: Gathers, ap: Aperture, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor,
                  w: int = 11, want_cube: bool = False, stream=None) -> dict:
    """CRS semblance search over the flattened A x B x C grid (include/seis.h:
    crs_semblance).  Returns best_idx, best_ABC [rows, 3], best_S, stack (and S)."""
    lib = load_library()
    dev = g.traces.device
    nA, nB, nC = int(A.numel()), int(B.numel()), int(C.numel())
    out = dict(best_idx=torch.empty(ap.rows, dtype=torch.int32, device=dev),
               best_ABC=torch.empty((ap.rows, 3), dtype=torch.float32, device=dev),
               best_S=torch.empty(ap.rows, dtype=torch.float32, device=dev),
               stack=torch.empty(ap.rows, dtype=torch.float32, device=dev))
    if want_cube:
        out["S"] = torch.empty((ap.rows, nA * nB * nC), dtype=torch.float32, device=dev)
    rc = lib.crs_semblance(ctypes.byref(g.descriptor()), ctypes.byref(ap.descriptor()),
                           _ptr(A), nA, _ptr(B), nB, _ptr(C), nC, w, _ptr(out.get("S")),
                           _ptr(out["best_idx"]), _ptr(out["best_ABC"]), _ptr(out["best_S"]),
                           _ptr(out["stack"]), _stream_handle(stream))
    _check(rc)
    return out


def search_variants() -> list[str]:
    """Names of the search kernel variants (index = variant id)."""
    lib = load_library()
    return [lib.seis_search_variant_name(i).decode() for i in range(lib.seis_search_variant_count())]


def set_search_variant(v: int) -> None:
    _check(load_library().seis_set_search_variant(int(v)))


def get_search_variant() -> int:
    return int(load_library().seis_get_search_variant())


def device_status(stream=None) -> None:
    """Raise if a kernel recorded a timed-out wait or an overflow since the last check."""
    _check(load_library().seis_device_status(_stream_handle(stream)))
