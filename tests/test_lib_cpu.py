"""libseis builds, loads and exports every entry point declared in include/seis.h; the
host-side argument checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1907_11678_gb300 import build as seis_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*"
                                r"([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = seis_build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for must in ("cmp_semblance", "crs_semblance", "seis_crs_aperture", "seis_last_error",
                 "seis_device_status"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def _err(lib):
    lib.seis_last_error.restype = ctypes.c_char_p
    return lib.seis_last_error().decode()


def test_null_descriptor_is_einval(lib):
    rc = lib.cmp_semblance(None, None, 1, 11, None, None, None, None, None, None)
    assert rc == -1 and "NULL" in _err(lib)


def test_even_window_is_einval(lib):
    from paper_1907_11678_gb300.seis import _Gathers
    fake = ctypes.c_void_p(16)               # never dereferenced: checks run first
    g = _Gathers(fake, fake, fake, None, fake, fake, fake, 1, 1, 10, 10)
    rc = lib.cmp_semblance(ctypes.byref(g), fake, ctypes.c_int32(3), ctypes.c_int32(4),
                           None, fake, None, fake, fake, None)
    assert rc == -1 and "odd" in _err(lib)
    rc = lib.cmp_semblance(ctypes.byref(g), fake, ctypes.c_int32(3), ctypes.c_int32(17),
                           None, fake, None, fake, fake, None)
    assert rc == -1


def test_trace_length_limit_is_einval(lib):
    from paper_1907_11678_gb300.seis import _Gathers
    fake = ctypes.c_void_p(16)
    g = _Gathers(fake, fake, fake, None, fake, fake, fake, 1, 1, 10, 20000)
    rc = lib.cmp_semblance(ctypes.byref(g), fake, ctypes.c_int32(3), ctypes.c_int32(11),
                           None, fake, None, fake, fake, None)
    assert rc == -1 and "max_trace_samples" in _err(lib)


def test_crs_needs_midpoints(lib):
    from paper_1907_11678_gb300.seis import _Aperture, _Gathers
    fake = ctypes.c_void_p(16)
    g = _Gathers(fake, fake, fake, None, fake, fake, fake, 1, 1, 10, 10)
    ap = _Aperture(fake, fake, fake, fake, fake, 1, 10, 0)
    rc = lib.crs_semblance(ctypes.byref(g), ctypes.byref(ap), fake, 1, fake, 1, fake, 1, 11,
                           None, fake, None, fake, fake, None)
    assert rc == -1 and "midpoint" in _err(lib)


def test_misaligned_traces_is_einval(lib):
    from paper_1907_11678_gb300.seis import _Gathers
    fake = ctypes.c_void_p(16)
    g = _Gathers(ctypes.c_void_p(18), fake, fake, None, fake, fake, fake, 1, 1, 10, 10)
    rc = lib.cmp_semblance(ctypes.byref(g), fake, ctypes.c_int32(3), ctypes.c_int32(11),
                           None, fake, None, fake, fake, None)
    assert rc == -1 and "aligned" in _err(lib)
