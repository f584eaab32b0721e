"""Batched search of uneven CMP gathers and CRS supergathers in one persistent launch."""
import numpy as np
import pytest

import oracle
from paper_1907_11678_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def seis():
    from paper_1907_11678_gb300 import build, seis as s
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return s


@pytest.fixture(scope="module")
def small(seis):
    ds, items, A, B, C = synth.batch_workload(n_items=48, seed=9, fold=(3, 20), ns=(120, 500),
                                              nc_range=(20, 45), crs_grid=(5, 3, 7))
    g = seis.to_device(ds)
    b = seis.batch_to_device(items, A, B, C, ds["out_rows"])
    return ds, items, A, B, C, g, b


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _item_ds(ds, it):
    """The item's traces as a one-gather dataset (input slicing only)."""
    tb, te = int(it["trace_begin"]), int(it["trace_end"])
    off = ds["trace_off"][tb:te + 1]
    return dict(traces=ds["traces"][off[0]:off[-1]], trace_off=off - off[0],
                h=ds["h"][tb:te], m=ds["m"][tb:te], gather_off=np.array([0, te - tb], np.int64),
                out_off=np.array([0, int(it["rows"])], np.int64),
                dt=np.float32([it["dt"]]))


def test_batch_matches_oracle_per_item(seis, small):
    ds, items, A, B, C, g, b = small
    got = _host(seis.batch_semblance(g, b, w=11, mode=0))
    torch.cuda.synchronize()
    seis.device_status()
    kinds = set()
    for it in items:
        r0, rows = int(it["out_begin"]), int(it["rows"])
        sub = _item_ds(ds, it)
        Ci = C[int(it["c_off"]):int(it["c_off"]) + int(it["nC"])]
        if it["kind"] == 0:
            ref = oracle.cmp_semblance(sub, Ci, w=11)
        else:
            nb = (np.array([0, len(sub["h"])], np.int64), np.arange(len(sub["h"]), dtype=np.int32),
                  np.float32([it["m_c"]]), np.array([0, rows], np.int64), np.float32([it["dt"]]))
            ref = oracle.crs_semblance(sub, nb, A, B, Ci, w=11, want_cube=True)
        kinds.add(int(it["kind"]))
        sl = slice(r0, r0 + rows)
        parity.check_picks(got["best_idx"][sl], got["best_S"][sl], got["stack"][sl], ref,
                           f"batch item {r0}")
    assert kinds == {0, 1}


def test_batch_modes_and_single_kernels_agree_bitwise(seis, small):
    """The persistent launch, one launch per item, and the plain CMP / CRS search kernels
    (through apertures = the items' own traces) give bit-identical results."""
    ds, items, A, B, C, g, b = small
    p = _host(seis.batch_semblance(g, b, w=11, mode=0))
    q = _host(seis.batch_semblance(g, b, w=11, mode=1))
    for k in p:
        np.testing.assert_array_equal(p[k], q[k])
    t = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    for it in items[:12]:
        r0, rows = int(it["out_begin"]), int(it["rows"])
        sub = seis.to_device(_item_ds(ds, it))
        Ci = C[int(it["c_off"]):int(it["c_off"]) + int(it["nC"])]
        if it["kind"] == 0:
            o = _host(seis.cmp_semblance(sub, t(Ci), w=11))
        else:
            ap = seis.crs_aperture(sub, [0], 1e9)
            ap.m_c.fill_(float(it["m_c"]))
            o = _host(seis.crs_semblance(sub, ap, t(A), t(B), t(Ci), w=11))
        np.testing.assert_array_equal(o["best_idx"], p["best_idx"][r0:r0 + rows])
        np.testing.assert_array_equal(o["best_S"], p["best_S"][r0:r0 + rows])
        np.testing.assert_array_equal(o["stack"], p["stack"][r0:r0 + rows])


def test_batch_cuda_graph_replay(seis, small):
    ds, items, A, B, C, g, b = small
    out = seis.batch_semblance(g, b, w=11, mode=0)            # warm-up outside capture
    torch.cuda.synchronize()
    ref = _host(out)
    for v in out.values():
        v.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        seis.batch_semblance(g, b, w=11, mode=0, out=out)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    seis.device_status()
    got = _host(out)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k])


def test_batch_skips_bad_item(seis, small):
    ds, items, A, B, C, g, b = small
    bad = items.copy()
    bad[3]["trace_end"] = 10 ** 9                              # out of range: skipped
    bb = seis.batch_to_device(bad, A, B, C, ds["out_rows"])
    seis.batch_semblance(g, bb, w=11, mode=0)
    with pytest.raises(seis.SeisError):
        seis.device_status()
    seis.device_status()                                       # cleared


def test_batch_autotune_picks_a_built_variant_and_keeps_results(seis, small):
    ds, items, A, B, C, g, b = small
    ref = _host(seis.batch_semblance(g, b, w=11, mode=0))
    chosen, ms = seis.autotune_batch(g, b, w=11, reps=1)
    assert chosen in (0, 1, 3, 4, 9, 10)
    assert ms[chosen] > 0 and all(ms[v] > 0 for v in (0, 1, 3, 4, 9, 10))
    assert all(ms[v] == -1 for v in range(len(ms)) if v not in (0, 1, 3, 4, 9, 10))
    got = _host(seis.batch_semblance(g, b, w=11, mode=0))     # runs the chosen variant
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k])
    seis.autotune_clear()


def test_batch_workload_distributions_sampled(seis):
    """300 items drawn from the batch workload's own distributions (fold 8-120, 1000-4000
    samples at 2 or 4 ms, 101-201 C or an 11 x 11 x 21 CRS grid); the oracle checks seeded
    rows of a seeded sample of items of both kinds."""
    ds, items, A, B, C = synth.batch_workload(n_items=300, seed=41)
    g = seis.to_device(ds)
    b = seis.batch_to_device(items, A, B, C, ds["out_rows"])
    got = _host(seis.batch_semblance(g, b, w=11, mode=0))
    torch.cuda.synchronize()
    seis.device_status()
    rng = np.random.default_rng(42)
    kinds = set()
    for idx in rng.choice(len(items), 8, replace=False):
        it = items[idx]
        r0, rows = int(it["out_begin"]), int(it["rows"])
        sub = _item_ds(ds, it)
        sel = np.sort(rng.choice(rows, min(rows, 12), replace=False))
        Ci = C[int(it["c_off"]):int(it["c_off"]) + int(it["nC"])]
        if it["kind"] == 0:
            ref = oracle.cmp_semblance(sub, Ci, w=11, rows=sel)
        else:
            Ai = A[int(it["a_off"]):int(it["a_off"]) + int(it["nA"])]
            Bi = B[int(it["b_off"]):int(it["b_off"]) + int(it["nB"])]
            nb = (np.array([0, len(sub["h"])], np.int64), np.arange(len(sub["h"]), dtype=np.int32),
                  np.float32([it["m_c"]]), np.array([0, rows], np.int64), np.float32([it["dt"]]))
            ref = oracle.crs_semblance(sub, nb, Ai, Bi, Ci, w=11, rows=sel, want_cube=True)
        kinds.add(int(it["kind"]))
        parity.check_picks(got["best_idx"][r0 + sel], got["best_S"][r0 + sel],
                           got["stack"][r0 + sel], ref, f"batch workload item {idx}")
    assert kinds == {0, 1}
