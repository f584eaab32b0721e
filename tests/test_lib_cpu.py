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


def test_autotune_cache_roundtrip(lib, tmp_path):
    """The autotune table saves and loads as JSON without a GPU (host logic only)."""
    lib.seis_autotune_save.argtypes = [ctypes.c_char_p]
    lib.seis_autotune_load.argtypes = [ctypes.c_char_p]
    p = tmp_path / "tune.json"
    p.write_text('{"format": "seis-autotune-1", "entries": [\n'
                 '  {"crs": 0, "w": 11, "cand_bucket": 7, "rows_bucket": 10, "fold_bucket": 5, "variant": 3},\n'
                 '  {"crs": 1, "w": 11, "cand_bucket": 14, "rows_bucket": 10, "fold_bucket": 0, "variant": 1}\n]}\n')
    assert lib.seis_autotune_clear() == 0
    assert lib.seis_autotune_load(str(p).encode()) == 0
    out = tmp_path / "out.json"
    assert lib.seis_autotune_save(str(out).encode()) == 0
    txt = out.read_text()
    assert '"variant": 3' in txt and '"variant": 1' in txt and txt.count('"crs"') == 2
    bad = tmp_path / "bad.json"
    bad.write_text('{"entries": [{"crs": 0, "w": 11, "cand_bucket": 7, "rows_bucket": 10, '
                   '"fold_bucket": 5, "variant": 99}]}')
    assert lib.seis_autotune_load(str(bad).encode()) == -1
    assert lib.seis_autotune_clear() == 0


def test_variant_selector(lib):
    n = lib.seis_search_variant_count()
    assert n >= 5
    default = lib.seis_get_search_variant()
    assert default == 4                          # the packed 15 x 2 shape until changed
    assert lib.seis_set_search_variant(n) == -1
    assert lib.seis_set_search_variant(-1) == -1
    assert lib.seis_set_search_variant(0) == 0 and lib.seis_get_search_variant() == 0
    assert lib.seis_set_search_variant(default) == 0
    # every variant has its own name; the scheduler-balanced 12-warp shape is among them
    lib.seis_search_variant_name.restype = ctypes.c_char_p
    lib.seis_search_variant_name.argtypes = [ctypes.c_int]
    names = [lib.seis_search_variant_name(v).decode() for v in range(n)]
    assert all(names) and len(set(names)) == n
    assert lib.seis_search_variant_name(n).decode() == ""
    assert any(nm.startswith("12 warps x 2 candidates, packed") for nm in names)


def test_refine_starts_arguments_are_checked(lib):
    fake = ctypes.c_void_p(16)               # never dereferenced: checks run first
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    # more starts than candidates
    rc = lib.crs_top_starts(fake, i64(10), fake, i32(2), fake, i32(1), fake, i32(3), i32(7),
                            fake, None)
    assert rc == -1 and "nstart" in _err(lib)
    rc = lib.crs_top_starts(fake, i64(10), fake, i32(2), fake, i32(1), fake, i32(3), i32(0),
                            fake, None)
    assert rc == -1
    rc = lib.crs_top_starts(None, i64(10), fake, i32(2), fake, i32(1), fake, i32(3), i32(1),
                            fake, None)
    assert rc == -1 and "NULL" in _err(lib)
    lib.seis_refine_multi_workspace_size.restype = ctypes.c_size_t
    lib.seis_refine_workspace_size.restype = ctypes.c_size_t
    assert lib.seis_refine_multi_workspace_size(i64(1000)) > lib.seis_refine_workspace_size(i64(1000))
    rc = lib.crs_refine_multi(None, None, fake, i32(0), None, None, i32(20), ctypes.c_float(0.05),
                              i32(11), fake, fake, fake, fake, fake, ctypes.c_size_t(0),
                              i64(10), None)
    assert rc == -1 and "nstart" in _err(lib)


def test_pragmatic_and_offset_aperture_arguments(lib):
    fake = ctypes.c_void_p(16)
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    rc = lib.crs_pragmatic(fake, None, fake, fake, fake, i32(1), fake, i32(1), fake, i32(1),
                           ctypes.c_float(0.0), i32(11), fake, fake, fake, fake,
                           ctypes.c_size_t(0), i64(10), None)
    assert rc == -1 and "aperture" in _err(lib)
    lib.seis_pragmatic_workspace_size.restype = ctypes.c_size_t
    assert lib.seis_pragmatic_workspace_size(i64(100)) >= 100 * 52


# --- the binding refuses malformed arrays on the host, before any kernel could read them ----

@pytest.fixture(scope="module")
def host_gathers(lib):
    import torch
    from paper_1907_11678_gb300 import seis, synth
    ds = synth.crs_line(6, 4, 200, 0.004, 0.0, 500.0, 1, 0, None, seed=21)
    return seis, torch, seis.to_device(ds, device="cpu")


def test_binding_refuses_short_operator_arrays(host_gathers):
    seis, torch, g = host_gathers
    with pytest.raises(ValueError, match="params"):
        seis.stack(g, None, torch.zeros(g.rows - 1))


def test_binding_refuses_wrong_output_arrays(host_gathers):
    seis, torch, g = host_gathers
    C = torch.ones(5)
    good = dict(best_idx=torch.zeros(g.rows, dtype=torch.int32),
                best_S=torch.zeros(g.rows), stack=torch.zeros(g.rows))
    for key, bad in (("best_idx", torch.zeros(g.rows)),                       # dtype
                     ("best_S", torch.zeros(g.rows - 1)),                     # size
                     ("stack", torch.zeros(2 * g.rows)[::2]),                 # layout
                     ("S", torch.zeros(g.rows, 4))):                          # cube size
        out = dict(good, **{key: bad})
        with pytest.raises(ValueError, match=key):
            seis.cmp_semblance(g, C, out=out)
    with pytest.raises(ValueError, match="required"):
        seis.cmp_semblance(g, C, out={"best_idx": good["best_idx"]})


def test_binding_refuses_mis_shaped_cube_and_starts(host_gathers):
    seis, torch, g = host_gathers
    A, B, C = torch.zeros(3), torch.zeros(2), torch.zeros(4)
    with pytest.raises(ValueError, match="S_cube"):
        seis.crs_top_starts(torch.zeros(10, 23), A, B, C, 2)
    ap = seis.Aperture(*(torch.zeros(1),) * 5, n_central=1, max_rows=200, rows=200)
    with pytest.raises(ValueError, match="starts"):
        seis.crs_refine_multi(g, ap, torch.zeros(2, 199, 3), (0, 0, 0), (1, 1, 1))



def test_missing_library_fails_loudly(tmp_path):
    """With libseis.so absent the binding raises on the first call: there is no CPU
    fallback to take its place."""
    import subprocess
    import sys
    code = (
        "from paper_1907_11678_gb300 import build, seis, synth\n"
        f"build.LIB = {str(tmp_path / 'libseis.so')!r}\n"
        "ds = synth.crs_line(3, 4, 200, 0.004, 0.0, 500.0, 1, 0, None, seed=22)\n"
        "g = seis.to_device(ds, device='cpu')\n"
        "try:\n"
        "    seis.cmp_semblance(g, seis.velocity_grid(1400.0, 4500.0, 5, device='cpu'))\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    print('no error')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert "raised: libseis.so not found" in r.stdout


def test_binding_refuses_inconsistent_offsets(host_gathers):
    """The kernels index through the offset arrays, so to_device refuses offsets that do not
    index inside the dataset's own arrays."""
    seis, torch, _ = host_gathers
    from paper_1907_11678_gb300 import synth
    ds = synth.crs_line(4, 4, 200, 0.004, 0.0, 500.0, 1, 0, None, seed=23)
    seis.to_device(ds, device="cpu")                                   # consistent: accepted
    bad = []
    t = ds["trace_off"].copy(); t[-1] += 1; bad.append(("trace_off", dict(ds, trace_off=t)))
    t = ds["trace_off"].copy(); t[2], t[3] = t[3], t[2]; bad.append(("trace_off", dict(ds, trace_off=t)))
    g = ds["gather_off"].copy(); g[-1] += 1; bad.append(("gather_off", dict(ds, gather_off=g)))
    o = ds["out_off"].copy(); o[1] = -1; bad.append(("out_off", dict(ds, out_off=o)))
    bad.append(("out_off", dict(ds, out_off=ds["out_off"][:-1])))
    bad.append(("h", dict(ds, h=ds["h"][:-1])))
    bad.append(("dt", dict(ds, dt=ds["dt"][:-1])))
    for name, d in bad:
        with pytest.raises(ValueError, match=name):
            seis.to_device(d, device="cpu")
