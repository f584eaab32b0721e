"""Every search-kernel variant (tile shape; scalar, packed or hybrid FP32 arithmetic) on the
GPU: each sums in the same order, so all must give the same bits, and those bits match the
FP64 oracle.  The full-size workloads also run here in the benchmark's launch configuration
(the variant the autotuner picks on the benchmark's tuning slice)."""
import numpy as np
import pytest

import oracle
from paper_1907_11678_gb300 import synth
from tests import parity
from tests.dsutil import dataset

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def seis():
    from paper_1907_11678_gb300 import build, seis as s
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return s


def _host(out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _every_variant(seis, run):
    """run() under each variant in turn (no autotuned entry may override the choice)."""
    names = seis.search_variants()
    default = seis.get_search_variant()
    seis.autotune_clear()
    outs = []
    try:
        for v in range(len(names)):
            seis.set_search_variant(v)
            outs.append(_host(run()))
            seis.device_status()
    finally:
        seis.set_search_variant(default)
    return names, outs


def _assert_bit_identical(names, outs):
    for v in range(1, len(outs)):
        for k in outs[0]:
            np.testing.assert_array_equal(outs[v][k], outs[0][k],
                                          err_msg=f"variant {v} ({names[v]}): {k}")


def _ragged_cmp():
    """Gathers of different fold (one of 37 traces: two stages), output length and dt;
    traces of different lengths; an empty gather and a fold-1 gather."""
    rng = np.random.default_rng(17)
    traces, h, sizes, outs, dts = [], [], [], [], []
    for fold, ns, dt in [(37, 333, 0.004), (0, 40, 0.004), (1, 130, 0.002), (9, 77, 0.002)]:
        for i in range(fold):
            L = ns + int(rng.integers(-20, 25)) if fold > 1 else ns
            traces.append(rng.standard_normal(max(L, 1)).astype(np.float32))
            h.append(rng.uniform(0, 1600))
        sizes.append(fold); outs.append(ns); dts.append(dt)
    ds = dataset(traces, h, 0.0, gather_sizes=sizes, out_ns=outs)
    ds["dt"] = np.float32(dts)
    return ds


@pytest.mark.parametrize("case", ["events", "ragged"])
def test_every_cmp_variant_bit_identical_and_matches_oracle(seis, case):
    """45 candidates: two candidate passes for every tile shape (28 or 30 per pass)."""
    if case == "events":
        ds = synth.cmp_line(3, 37, 420, 0.004, 0.0, 1800.0, 3, 1.5, seed=61)
    else:
        ds = _ragged_cmp()
    C = oracle.velocity_grid(1400.0, 4500.0, 45).astype(np.float32)
    g = seis.to_device(ds)
    Cd = torch.from_numpy(C).cuda()
    names, outs = _every_variant(seis, lambda: seis.cmp_semblance(g, Cd, w=11, want_cube=True))
    _assert_bit_identical(names, outs)
    ref = oracle.cmp_semblance(ds, C)
    parity.check_cube(outs[0]["S"], ref, f"variants cmp {case}")
    parity.check_picks(outs[0]["best_idx"], outs[0]["best_S"], outs[0]["stack"], ref,
                       f"variants cmp {case}")


def test_every_crs_variant_bit_identical_and_matches_oracle(seis):
    """Apertures of different size (a line end), 5 x 3 x 7 = 105 candidates (four passes)."""
    ds = synth.crs_line(9, 12, 300, 0.004, 0.0, 1500.0, 2, 1, 2.0, seed=62)
    central = [0, 4, 8]
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, central, 30.0)
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    A = oracle.linear_grid(alo, ahi, 5).astype(np.float32)
    B = oracle.linear_grid(blo, bhi, 3).astype(np.float32)
    C = oracle.linear_grid(clo, chi, 7).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    names, outs = _every_variant(
        seis, lambda: seis.crs_semblance(g, ap, t(A), t(B), t(C), w=11, want_cube=True))
    _assert_bit_identical(names, outs)
    ref = oracle.crs_semblance(ds, oracle.aperture(ds, central, 30.0), A, B, C, want_cube=True)
    parity.check_cube(outs[0]["S"], ref, "variants crs")
    parity.check_picks(outs[0]["best_idx"], outs[0]["best_S"], outs[0]["stack"], ref,
                       "variants crs")


@pytest.mark.slow
def test_cmp_line_full_size_in_the_benchmark_configuration(seis):
    """The CMP line at full size (4096 gathers x fold 60 x 2000 samples, 201 candidates,
    w = 11, no cube) with the variant the autotuner picks on the benchmark's 512-gather
    tuning slice; the oracle checks a seeded sample of rows."""
    ds = synth.workload_cmp_line()
    C = oracle.velocity_grid(1400.0, 4500.0, 201).astype(np.float32)
    Cd = torch.from_numpy(C).cuda()
    sub = synth.cmp_line(512, 60, 2000, 0.004, 25.0, 3000.0, 8, 1.0, seed=99,
                         v_range=(2550.0, 3450.0), v_gradient=0.5)
    seis.autotune_clear()
    try:
        chosen, _ = seis.autotune_cmp(seis.to_device(sub), Cd, w=11, reps=1)
        print(f"[parity] cmp-line variant {chosen}: {seis.search_variants()[chosen]}")
        got = _host(seis.cmp_semblance(seis.to_device(ds), Cd, w=11))
        seis.device_status()
    finally:
        seis.autotune_clear()
    rows = np.sort(np.random.default_rng(3).choice(int(ds["out_off"][-1]), 512, replace=False))
    ref = oracle.cmp_semblance(ds, C, rows=rows)
    rep = parity.check_picks(got["best_idx"][rows], got["best_S"][rows], got["stack"][rows],
                             ref, "cmp-line (bench variant)")
    assert rep["pick_agree"] > 0.98


@pytest.mark.slow
def test_crs_line_slice_in_the_benchmark_configuration(seis):
    """Two central CMPs of the CRS line (aperture 1008 traces, 1500 samples, 21 x 21 x 41)
    with the variant the autotuner picks on the benchmark's 4-central tuning slice."""
    ds = synth.workload_crs_line()
    g = seis.to_device(ds)
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    A = oracle.linear_grid(alo, ahi, 21).astype(np.float32)
    B = oracle.linear_grid(blo, bhi, 21).astype(np.float32)
    C = oracle.linear_grid(clo, chi, 41).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    central = ds["central"][[100, 900]]
    ap = seis.crs_aperture(g, central, ds["apm"])
    seis.autotune_clear()
    try:
        apt = seis.crs_aperture(g, ds["central"][:6], ds["apm"])
        chosen, _ = seis.autotune_crs(g, apt, t(A), t(B), t(C), w=11, reps=1)
        print(f"[parity] crs-line variant {chosen}: {seis.search_variants()[chosen]}")
        got = _host(seis.crs_semblance(g, ap, t(A), t(B), t(C), w=11))
        seis.device_status()
    finally:
        seis.autotune_clear()
    # most rows of this noisy line have near-ties (top-two gap < 1e-4), where any admissible
    # argmax is correct, so sample enough rows to hold a few dozen clear picks as well
    rows = np.sort(np.random.default_rng(4).choice(ap.rows, 96, replace=False))
    ref = oracle.crs_semblance(ds, oracle.aperture(ds, central, ds["apm"]), A, B, C,
                               rows=rows, want_cube=True)
    rep = parity.check_picks(got["best_idx"][rows], got["best_S"][rows], got["stack"][rows],
                             ref, "crs-line (bench variant)")
    assert rep["pick_agree"] >= 0.9 and rep["clear_rows"] > 0.1
