"""The allocation-free batched search (seis_batch_semblance_noalloc) against the batched
search with a caller workspace.

Callers that cannot allocate device memory where they call the library (a service under a
fixed device-memory budget, a plug-in whose host owns every allocation, a latency-bound
loop that cannot afford cudaMalloc's possible device synchronisation) use this entry point;
its scratch lives in a device array inside the library.  This file is collected last so
that a run stopping at the first failure has run every other test first; it must also pass
alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_1907_11678_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_workspace_entry_point_twice():
    from paper_1907_11678_gb300 import build, seis
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    lib = seis.load_library()
    lib.seis_batch_semblance_noalloc.restype = ctypes.c_int
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.seis_batch_semblance_noalloc.argtypes = [vp, vp, i64, vp, i32, vp, i32, vp, i32, i32,
                                                 vp, vp, vp, vp, i64, vp]
    ds, items, A, B, C = synth.batch_workload(n_items=40, seed=13, fold=(3, 18), ns=(150, 450),
                                              nc_range=(15, 40), crs_grid=(5, 3, 7))
    g = seis.to_device(ds)
    b = seis.batch_to_device(items, A, B, C, ds["out_rows"])
    ref = {k: v.cpu().numpy() for k, v in seis.batch_semblance(g, b, w=11, mode=0).items()}
    torch.cuda.synchronize()
    seis.device_status()
    rows = ds["out_rows"]
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):                                   # two calls in a row share the array
        out = dict(best_idx=torch.full((rows,), -7, dtype=torch.int32, device="cuda"),
                   best_ABC=torch.full((rows, 3), -7.0, device="cuda"),
                   best_S=torch.full((rows,), -7.0, device="cuda"),
                   stack=torch.full((rows,), -7.0, device="cuda"))
        rc = lib.seis_batch_semblance_noalloc(
            ctypes.byref(g.descriptor()), P(b.items), b.nitems, P(b.poolA), int(b.poolA.numel()),
            P(b.poolB), int(b.poolB.numel()), P(b.poolC), int(b.poolC.numel()), 11,
            P(out["best_idx"]), P(out["best_ABC"]), P(out["best_S"]), P(out["stack"]), rows,
            stream)
        assert rc == 0, lib.seis_last_error().decode()
        torch.cuda.synchronize()
        seis.device_status()
        for k in ref:
            np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k], err_msg=f"call {call}: {k}")


def _noalloc_fn(lib):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.seis_batch_semblance_noalloc.restype = ctypes.c_int
    lib.seis_batch_semblance_noalloc.argtypes = [vp, vp, i64, vp, i32, vp, i32, vp, i32, i32,
                                                 vp, vp, vp, vp, i64, vp]
    return lib.seis_batch_semblance_noalloc


def test_noalloc_takes_its_documented_maximum():
    """Exactly SEIS_NOALLOC_MAX_ITEMS tiny items (fold 1, 40 samples, 8 output rows, three C
    candidates each) are accepted and give the workspace entry point's results bit for bit."""
    from paper_1907_11678_gb300 import build, seis
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    lib = seis.load_library()
    fn = _noalloc_fn(lib)
    n, L, rows = 65536, 40, 8
    rng = np.random.default_rng(29)
    traces = rng.standard_normal(n * L).astype(np.float32)
    ds = dict(traces=traces, trace_off=np.arange(n + 1, dtype=np.int64) * L,
              h=rng.uniform(0.0, 60.0, n).astype(np.float32), m=np.zeros(n, np.float32),
              gather_off=np.array([0, n], np.int64), out_off=np.array([0, n * rows], np.int64),
              dt=np.float32([0.004]))
    items = np.zeros(n, synth.BATCH_ITEM_DTYPE)
    items["trace_begin"] = np.arange(n)
    items["trace_end"] = np.arange(n) + 1
    items["out_begin"] = np.arange(n) * rows
    items["rows"] = rows
    items["dt"] = 0.004
    items["nA"] = items["nB"] = 1
    items["nC"] = 3
    poolA = np.zeros(1, np.float32)
    poolB = np.zeros(1, np.float32)
    poolC = np.float32(4.0 / np.array([1500.0, 2500.0, 4000.0]) ** 2)
    g = seis.to_device(ds)
    b = seis.batch_to_device(items, poolA, poolB, poolC, n * rows)
    assert lib.seis_batch_workspace_size(n) == 524800
    ref = {k: v.cpu().numpy() for k, v in seis.batch_semblance(g, b, w=3, mode=0).items()}
    torch.cuda.synchronize()
    seis.device_status()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    out = dict(best_idx=torch.full((n * rows,), -7, dtype=torch.int32, device="cuda"),
               best_ABC=torch.full((n * rows, 3), -7.0, device="cuda"),
               best_S=torch.full((n * rows,), -7.0, device="cuda"),
               stack=torch.full((n * rows,), -7.0, device="cuda"))
    rc = fn(ctypes.byref(g.descriptor()), P(b.items), n, P(b.poolA), 1, P(b.poolB), 1,
            P(b.poolC), 3, 3, P(out["best_idx"]), P(out["best_ABC"]), P(out["best_S"]),
            P(out["stack"]), n * rows, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.seis_last_error().decode()
    torch.cuda.synchronize()
    seis.device_status()
    for k in ref:
        np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k], err_msg=k)
    assert (ref["best_S"] > 0).mean() > 0.5          # the rows were really searched


def test_noalloc_rejects_too_many_items():
    from paper_1907_11678_gb300 import seis
    lib = seis.load_library()
    lib.seis_batch_semblance_noalloc.restype = ctypes.c_int
    fake = ctypes.c_void_p(256)
    rc = lib.seis_batch_semblance_noalloc(fake, fake, ctypes.c_int64(65537), fake, 1, fake, 1,
                                          fake, 1, 11, fake, fake, fake, fake,
                                          ctypes.c_int64(1), None)
    assert rc == -1 and "at most" in lib.seis_last_error().decode()
