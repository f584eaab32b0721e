"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics, not by
the oracle itself (CPU only)."""
import json
import os

import math

import numpy as np
import pytest

import oracle
from paper_1907_11678_gb300 import synth
from tests.dsutil import dataset, pythagorean_offsets, spike_wavelet

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Eq. 1 worked example (hand-derived, tests/golden) ---------------------------------

def test_worked_example_golden():
    ex = json.load(open(os.path.join(GOLDEN, "cmp_worked_example.json")))
    ds = dataset(ex["traces"], ex["h"], ex["dt"])
    r = oracle.cmp_semblance(ds, np.array(ex["C"]), w=ex["w"], rows=[ex["row"]])
    np.testing.assert_allclose(r.S[0], ex["expect_S"], rtol=0, atol=1e-15)
    assert list(r.N[0]) == ex["expect_N"]
    assert r.best_idx[0] == ex["expect_best_idx"]
    assert r.stack[0] == pytest.approx(ex["expect_stack"], abs=1e-15)
    # stack at each candidate: one-candidate searches
    for c, want in enumerate(ex["expect_stack_per_candidate"]):
        rc = oracle.cmp_semblance(ds, np.array([ex["C"][c]]), w=ex["w"], rows=[ex["row"]])
        assert rc.stack[0] == pytest.approx(want, abs=1e-15)


# --- Eq. 1 closed forms and invariants ----------------------------------------------------

def _grid(nc=21):
    return oracle.velocity_grid(1400.0, 4500.0, nc)


def test_velocity_grid_closed_form():
    C = oracle.velocity_grid(1400.0, 4500.0, 5)
    v = np.array([1400.0, 2175.0, 2950.0, 3725.0, 4500.0])
    np.testing.assert_allclose(C, 4.0 / v ** 2, rtol=1e-15)
    assert oracle.velocity_grid(2000.0, 3000.0, 1)[0] == pytest.approx(1e-6)


def test_constant_traces_semblance_one():
    rng = np.random.default_rng(0)
    M, ns = 12, 300
    h = np.linspace(0, 1500, M)
    c0 = rng.uniform(0.5, 2.0)
    ds = dataset([np.full(ns, c0)] * M, h, 0.004)
    r = oracle.cmp_semblance(ds, _grid())
    has = r.N > 0
    assert has.any() and (~has).any()
    np.testing.assert_allclose(r.S[has], 1.0, atol=1e-14)
    assert np.all(r.S[~has] == 0.0)
    # unequal constants c_i, every trace taking part: S = (sum c)^2 / (N sum c^2)
    cs = rng.uniform(-1.0, 2.0, M).astype(np.float32).astype(np.float64)
    ds2 = dataset([np.full(ns, c) for c in cs], h, 0.004)
    r2 = oracle.cmp_semblance(ds2, _grid())
    full = r2.N == M
    assert full.sum() > 100
    np.testing.assert_allclose(r2.S[full], cs.sum() ** 2 / (M * (cs ** 2).sum()), rtol=1e-12)


def test_single_trace_semblance_one():
    rng = np.random.default_rng(1)
    ds = dataset([rng.standard_normal(400)], [800.0], 0.004)
    r = oracle.cmp_semblance(ds, _grid())
    one = r.N == 1
    np.testing.assert_allclose(r.S[one], 1.0, atol=1e-13)
    assert np.all(r.S[r.N == 0] == 0.0)


def test_zero_data():
    ds = dataset([np.zeros(200)] * 5, np.linspace(0, 1000, 5), 0.004)
    r = oracle.cmp_semblance(ds, _grid())
    assert np.all(r.S == 0.0) and np.all(r.stack == 0.0)


def test_random_bounds_cauchy_schwarz():
    ds = synth.cmp_line(3, 17, 500, 0.004, 0.0, 2000.0, 3, 0.5, seed=7)
    r = oracle.cmp_semblance(ds, _grid(31))
    assert r.S.min() >= 0.0 and r.S.max() <= 1.0 + 1e-12
    assert np.all(r.best_S >= r.second_S)



# --- symmetries of Eq. 1: the order of the traces and the scale of the amplitudes -------

def _permute_within_gathers(ds, seed):
    """The same gathers, each gather's traces (with their offsets and midpoints) in a
    random order."""
    rng = np.random.default_rng(seed)
    go, to = ds["gather_off"], ds["trace_off"]
    order = np.concatenate([go[g] + rng.permutation(go[g + 1] - go[g])
                            for g in range(len(go) - 1)]).astype(np.int64)
    pieces = [ds["traces"][to[i]:to[i + 1]] for i in order]
    off = np.zeros(len(order) + 1, np.int64)
    off[1:] = np.cumsum([len(a) for a in pieces])
    out = dict(ds, traces=np.concatenate(pieces), trace_off=off, h=ds["h"][order])
    if ds.get("m") is not None:
        out["m"] = ds["m"][order]
    return out


def _assert_same_search(a, b, atol=1e-12):
    np.testing.assert_array_equal(b.N, a.N)
    np.testing.assert_allclose(b.S, a.S, rtol=0, atol=atol)
    np.testing.assert_allclose(b.stack, a.stack, rtol=0, atol=atol)
    clear = a.best_S - a.second_S > 1e-9
    assert clear.mean() > 0.9
    np.testing.assert_array_equal(b.best_idx[clear], a.best_idx[clear])


def test_cmp_trace_order_invariance():
    """Eq. 1 sums over the traces of a gather, so their order changes S, the trace count,
    the pick and the stack by rounding only (a trace paired with another trace's offset, or
    a sum that leaves its gather, would not)."""
    ds = synth.cmp_line(3, 13, 400, 0.004, 0.0, 1800.0, 3, 1.0, seed=31)
    C = _grid(23)
    _assert_same_search(oracle.cmp_semblance(ds, C),
                        oracle.cmp_semblance(_permute_within_gathers(ds, 32), C))


def test_crs_aperture_order_invariance():
    """The CRS sums run over the aperture's traces: listing them in another order (and
    reordering the traces of every CMP in the line) changes nothing beyond rounding."""
    ds = synth.crs_line(9, 8, 300, 0.004, 0.0, 1200.0, 2, 1, 2.0, seed=33)
    A = np.float32([-3e-4, 0.0, 2e-4]); B = np.float32([-1e-6, 0.0, 1e-6])
    C = np.float32(_grid(5))
    central = [3, 4, 5]
    nb = oracle.aperture(ds, central, 37.5)
    a = oracle.crs_semblance(ds, nb, A, B, C, want_cube=True)
    rng = np.random.default_rng(34)
    off, tr = nb[0], nb[1].copy()
    for i in range(len(central)):
        tr[off[i]:off[i + 1]] = rng.permutation(tr[off[i]:off[i + 1]])
    b = oracle.crs_semblance(ds, (off, tr) + tuple(nb[2:]), A, B, C, want_cube=True)
    _assert_same_search(a, b)
    p = _permute_within_gathers(ds, 35)
    _assert_same_search(a, oracle.crs_semblance(p, oracle.aperture(p, central, 37.5),
                                                A, B, C, want_cube=True))


def test_amplitude_scale_is_exact():
    """S is a ratio of two quadratic forms in the amplitudes and the stack is linear in
    them: scaling every trace by -4 (a power of two, so every FP64 step scales exactly)
    leaves S and the pick bit-identical and scales the stack by exactly -4."""
    ds = synth.cmp_line(2, 11, 300, 0.004, 0.0, 1500.0, 3, 2.0, seed=36)
    C = _grid(17)
    a = oracle.cmp_semblance(ds, C)
    b = oracle.cmp_semblance(dict(ds, traces=np.float32(-4.0) * ds["traces"]), C)
    np.testing.assert_array_equal(b.S, a.S)
    np.testing.assert_array_equal(b.best_idx, a.best_idx)
    np.testing.assert_array_equal(b.stack, -4.0 * a.stack)


# --- an exactly sampled hyperbolic event: S = 1 at the true C, argmax = true C ---------

def _exact_hyperbola(n0=240, ns=700, hw=5):
    dt = 1.0 / 256.0
    Ct = 2.0 ** -20                       # C h^2 / dt^2 = (4a)^2 for h = 16 a
    trip = [(0, n0)] + pythagorean_offsets(n0, 150)
    traces, h = [], []
    for a, mm in trip:
        traces.append(spike_wavelet(ns, mm, 2.5))
        h.append(16.0 * a)
    return dataset(traces, h, dt), Ct, len(trip)


def test_exact_hyperbola_semblance_one():
    ds, Ct, M = _exact_hyperbola()
    assert M >= 6
    grid = Ct * np.array([0.5, 0.8, 0.9, 1.0, 1.1, 1.25, 1.6])
    r = oracle.cmp_semblance(ds, grid, w=11, rows=[240])
    assert r.N[0, 3] == M
    assert r.S[0, 3] == pytest.approx(1.0, abs=1e-14)
    assert r.best_idx[0] == 3
    assert r.S[0, [0, 1, 2, 4, 5, 6]].max() < 0.99


# --- pure-Python brute force on tiny inputs (independent loop nest) ----------------------

def _brute_cmp(traces, h, dt, C, w, ns_out):
    hw = w // 2
    S = np.zeros((ns_out, len(C)))
    for n in range(ns_out):
        t0 = n * float(dt)
        for c, Cc in enumerate(C):
            Cc = float(Cc)
            num = [0.0] * w
            den = 0.0
            N = 0
            for f, hh in zip(traces, h):
                f = [float(a) for a in f]
                u = (t0 * t0 + Cc * float(hh) * float(hh)) ** 0.5 / float(dt)
                k = int(np.floor(u))
                if k - hw < 0 or k + hw + 1 > len(f) - 1:
                    continue
                x = u - k
                for j in range(-hw, hw + 1):
                    v = (f[k + j + 1] - f[k + j]) * x + f[k + j]
                    num[j + hw] += v
                    den += v * v
                N += 1
            S[n, c] = sum(a * a for a in num) / (N * den) if N and den > 0 else 0.0
    return S


@pytest.mark.parametrize("w", [1, 3, 5])
def test_bruteforce_tiny(w):
    rng = np.random.default_rng(w)
    traces = [rng.standard_normal(37).astype(np.float32) for _ in range(4)]
    traces.append(rng.standard_normal(29).astype(np.float32))          # a shorter trace
    h = np.float32([0.0, 110.0, 260.0, 420.0, 333.0])
    dt = np.float32(0.004)
    C = np.float32(oracle.velocity_grid(1400.0, 4500.0, 6))
    ds = dataset(traces, h, dt)
    r = oracle.cmp_semblance(ds, C, w=w)
    ref = _brute_cmp(traces, h, dt, C, w, len(traces[0]))
    np.testing.assert_allclose(r.S, ref, rtol=1e-12, atol=1e-14)


def test_multi_gather_rows_subset_matches_full():
    ds = synth.cmp_line(4, 9, 300, 0.004, 0.0, 1200.0, 2, 2.0, seed=3)
    C = _grid(11)
    full = oracle.cmp_semblance(ds, C)
    rows = np.array([0, 5, 299, 300, 301, 777, 1199])
    sub = oracle.cmp_semblance(ds, C, rows=rows)
    np.testing.assert_array_equal(sub.S, full.S[rows])
    np.testing.assert_array_equal(sub.best_idx, full.best_idx[rows])


# --- stack of a single trace: window mean of numpy.interp --------------------------------

def test_single_trace_stack_is_window_mean():
    rng = np.random.default_rng(5)
    ns, dt, hh, w = 300, 0.004, 700.0, 11
    f = rng.standard_normal(ns).astype(np.float32)
    ds = dataset([f], [hh], dt)
    C = _grid(9)
    r = oracle.cmp_semblance(ds, C, w=w)
    hw = w // 2
    for n in range(0, ns, 7):
        c = r.best_idx[n]
        u = np.sqrt((n * np.float64(np.float32(dt))) ** 2 + np.float64(np.float32(C[c]))
                    * np.float64(np.float32(hh)) ** 2) / np.float64(np.float32(dt))
        k = np.floor(u)
        if k - hw < 0 or k + hw + 1 > ns - 1:
            assert r.stack[n] == 0.0
            continue
        want = np.interp(u + np.arange(-hw, hw + 1), np.arange(ns), f.astype(np.float64)).mean()
        assert r.stack[n] == pytest.approx(want, rel=1e-12, abs=1e-14)


# --- CRS: reductions to CMP, an exactly sampled dipping plane, the aperture ---------------

def test_crs_with_zero_dm_equals_cmp():
    ds = synth.cmp_line(3, 10, 400, 0.004, 0.0, 1500.0, 3, 2.0, seed=11)
    C = np.float32(_grid(7))
    A = np.float32([-3e-4, 0.0, 2e-4])
    B = np.float32([-1e-6, 5e-7])
    nb = oracle.cmp_as_crs(ds)           # each gather is its own aperture: dm = 0
    cr = oracle.crs_semblance(ds, nb, A, B, C, want_cube=True)
    cm = oracle.cmp_semblance(ds, C)
    cube = cr.S.reshape(-1, len(A), len(B), len(C))
    for ia in range(len(A)):
        for ib in range(len(B)):
            np.testing.assert_array_equal(cube[:, ia, ib, :], cm.S)


def test_crs_flat_identical_cmps_equals_cmp():
    one = synth.cmp_line(1, 8, 300, 0.004, 0.0, 1200.0, 2, 2.0, seed=12)
    K = 5
    traces = [one["traces"][one["trace_off"][i]:one["trace_off"][i + 1]] for i in range(8)] * K
    h = np.tile(one["h"], K)
    m = np.repeat(np.arange(K) * 12.5, 8)
    ds = dataset(traces, h, 0.004, m=m, gather_sizes=[8] * K)
    nb = oracle.neighbours(ds, [2], 30.0)
    assert nb[0][-1] == 40
    out_off_c = np.array([0, 300], np.int64)
    C = np.float32(_grid(9))
    cr = oracle.crs_semblance(ds, (*nb, out_off_c, np.float32([0.004])), [0.0], [0.0], C,
                              want_cube=True)
    cm = oracle.cmp_semblance(one, C)
    np.testing.assert_allclose(cr.S, cm.S, rtol=1e-12, atol=1e-14)


def _exact_plane(n0=260, ns=700):
    """Traces whose CRS traveltime with A = 2^-6, B = 0, C = 2^-20 (dt = 1/256) lands on
    integer samples: u^2 = (n0 + 4 dm)^2 + (4 a)^2 (a Pythagorean triple per dm)."""
    dt = 1.0 / 256.0
    traces, h, m = [], [], []
    for dm in range(-3, 4):
        p = n0 + 4 * dm
        for a, mm in [(0, p)] + pythagorean_offsets(p, 90)[:6]:
            traces.append(spike_wavelet(ns, mm, 2.5))
            h.append(16.0 * a)
            m.append(100.0 + dm)
    ds = dataset(traces, h, dt, m=m, gather_sizes=[len(traces)])
    return ds, (2.0 ** -6, 0.0, 2.0 ** -20)


def test_crs_exact_dipping_plane():
    ds, (At, Bt, Ct) = _exact_plane()
    nb = (np.array([0, len(ds["h"])], np.int64), np.arange(len(ds["h"]), dtype=np.int32),
          np.float32([100.0]), np.array([0, 700], np.int64), np.float32([1.0 / 256]))
    A = At * np.array([0.5, 1.0, 1.5]); B = np.array([-2.0 ** -10, 0.0, 2.0 ** -10])
    C = Ct * np.array([0.8, 1.0, 1.2])
    r = oracle.crs_semblance(ds, nb, A, B, C, rows=[260], want_cube=True)
    true = (1 * 3 + 1) * 3 + 1
    assert r.N[0, true] == len(ds["h"])
    assert r.S[0, true] == pytest.approx(1.0, abs=1e-14)
    assert r.best_idx[0] == true
    assert np.delete(r.S[0], true).max() < 0.999


def test_crs_exact_B_term():
    """u^2 = (n0 + 4 dm)^2 + 4 dm^2 + (4a)^2 with A = 2^-6, B = 2^-14, C = 2^-20, dt = 1/256."""
    n0, ns, dt = 240, 700, 1.0 / 256.0
    traces, h, m = [], [], []
    for dm in range(-20, 21):
        p = n0 + 4 * dm
        for a in range(0, 150):
            mm2 = p * p + 4 * dm * dm + 16 * a * a
            r = int(round(np.sqrt(mm2)))
            if r * r == mm2 and r < ns - 10:
                traces.append(spike_wavelet(ns, r, 2.5)); h.append(16.0 * a); m.append(50.0 + dm)
    assert len(traces) >= 40 and len(set(m)) >= 20
    ds = dataset(traces, h, dt, m=m)
    nb = (np.array([0, len(h)], np.int64), np.arange(len(h), dtype=np.int32), np.float32([50.0]),
          np.array([0, ns], np.int64), np.float32([dt]))
    A = np.array([2.0 ** -6]); B = 2.0 ** -14 * np.array([0.0, 0.5, 1.0, 2.0]); C = [2.0 ** -20]
    r = oracle.crs_semblance(ds, nb, A, B, C, rows=[n0], want_cube=True)
    assert r.N[0, 2] == len(traces)
    assert r.S[0, 2] == pytest.approx(1.0, abs=1e-14)
    assert r.best_idx[0] == 2
    assert np.delete(r.S[0], 2).max() < 0.999


def test_neighbours_bruteforce():
    ds = synth.crs_line(30, 4, 200, 0.004, 0.0, 500.0, 1, 0, None, seed=2)
    central = np.array([0, 7, 15, 29], np.int32)
    off, tr, mc = oracle.neighbours(ds, central, 37.5)
    for c, g in enumerate(central):
        mg = ds["m"][ds["gather_off"][g]]
        want = np.nonzero(np.abs(ds["m"].astype(np.float64) - mg) <= 37.5)[0]
        np.testing.assert_array_equal(tr[off[c]:off[c + 1]], want)
        assert mc[c] == mg
    assert off[2] - off[1] == 7 * 4          # interior: +-3 CMPs


# --- gradient: central finite differences -------------------------------------------------

def test_gradient_matches_finite_differences():
    ds = synth.crs_line(9, 12, 600, 0.004, 0.0, 1500.0, 2, 1, 4.0, seed=21)
    nb = oracle.neighbours(ds, [4], 50.0)
    nbf = (*nb, np.array([0, 600], np.int64), np.float32([0.004]))
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    rng = np.random.default_rng(0)
    rows = np.arange(150, 560, 37)
    theta = np.stack([rng.uniform(alo, ahi, len(rows)) * 0.5,
                      rng.uniform(blo, bhi, len(rows)) * 0.5,
                      rng.uniform(clo, chi * 0.5, len(rows))], axis=1)
    base = oracle.crs_eval(ds, nbf, theta, rows=rows)
    scale = np.array([ahi - alo, bhi - blo, chi - clo])
    checked = 0
    for a in range(3):
        fd = {}
        for hrel in (1e-6, 2.5e-7):
            hstep = hrel * scale[a]
            tp = theta.copy(); tp[:, a] += hstep
            tm = theta.copy(); tm[:, a] -= hstep
            fd[hrel] = (oracle.crs_eval(ds, nbf, tp, rows=rows).S
                        - oracle.crs_eval(ds, nbf, tm, rows=rows).S) / (2 * hstep)
        smooth = np.abs(fd[1e-6] - fd[2.5e-7]) <= 1e-7 * (np.abs(fd[1e-6]) + 1e-3 / scale[a])
        g = base.grad[:, a]
        err = np.abs(g - fd[1e-6]) / (np.abs(fd[1e-6]) + 1e-3 / scale[a])
        assert np.all(err[smooth] < 1e-6), (a, err[smooth].max())
        checked += smooth.sum()
    assert checked >= 20


def test_eval_matches_search_at_grid_point():
    ds = synth.crs_line(7, 10, 500, 0.004, 0.0, 1500.0, 2, 1, 2.0, seed=31)
    nb = oracle.neighbours(ds, [3], 40.0)
    nbf = (*nb, np.array([0, 500], np.int64), np.float32([0.004]))
    A = np.float32([-2e-4, 0.0, 3e-4]); B = np.float32([0.0, 1e-6]); C = np.float32(_grid(5))
    rows = np.arange(100, 480, 41)
    s = oracle.crs_semblance(ds, nbf, A, B, C, rows=rows, want_cube=True)
    ia, ib, ic = 2, 1, 3
    th = np.tile(np.float64([A[ia], B[ib], C[ic]]), (len(rows), 1))
    e = oracle.crs_eval(ds, nbf, th, rows=rows)
    np.testing.assert_allclose(e.S, s.S[:, (ia * 2 + ib) * 5 + ic], rtol=1e-13, atol=1e-15)


# --- refinement invariants (reading c16; beyond these the result is unpinned) ------------

def test_refine_invariants_and_exact_plane():
    ds, (At, Bt, Ct) = _exact_plane()
    nb = (np.array([0, len(ds["h"])], np.int64), np.arange(len(ds["h"]), dtype=np.int32),
          np.float32([100.0]), np.array([0, 700], np.int64), np.float32([1.0 / 256]))
    lo = np.array([0.0, -2.0 ** -16, 0.5 * Ct]); hi = np.array([2.0 * At, 2.0 ** -16, 2.0 * Ct])
    rows = np.array([259, 260, 261])
    start = np.tile([At * 1.02, 2.0 ** -19, Ct * 0.99], (3, 1))
    r0 = oracle.crs_refine(ds, nb, start, lo, hi, steps=0, rows=rows)
    np.testing.assert_array_equal(r0.theta, start)
    r = oracle.crs_refine(ds, nb, start, lo, hi, steps=40, step0=0.01, rows=rows)
    assert np.all(r.S >= r0.S)
    assert np.all(r.theta >= lo) and np.all(r.theta <= hi)
    assert r.S[1] > 0.999


def test_top_starts_hand_worked():
    """Candidates ordered by S descending, lowest index first on ties; cand = (ia*nB+ib)*nC+ic."""
    S = np.array([[0.2, 0.5, 0.5, 0.1], [0.0, 0.0, 0.0, 0.0], [0.1, 0.2, 0.3, 0.4]])
    A, B, C = [1.0, 2.0], [10.0], [100.0, 200.0]
    got = oracle.top_starts(S, A, B, C, 3)
    want = np.array([[[1, 10, 200], [1, 10, 100], [2, 10, 200]],
                     [[2, 10, 100], [1, 10, 200], [2, 10, 100]],
                     [[1, 10, 100], [2, 10, 100], [1, 10, 200]]], np.float64)
    np.testing.assert_array_equal(got, want)


def test_refine_multi_keeps_best_start():
    ds, (At, Bt, Ct) = _exact_plane()
    nb = (np.array([0, len(ds["h"])], np.int64), np.arange(len(ds["h"]), dtype=np.int32),
          np.float32([100.0]), np.array([0, 700], np.int64), np.float32([1.0 / 256]))
    lo = np.array([0.0, -2.0 ** -16, 0.5 * Ct]); hi = np.array([2.0 * At, 2.0 ** -16, 2.0 * Ct])
    rows = np.array([259, 260, 261])
    starts = np.stack([np.tile([At * 1.6, 2.0 ** -18, Ct * 1.7], (3, 1)),
                       np.tile([At * 1.02, 2.0 ** -19, Ct * 0.99], (3, 1))])
    single = [oracle.crs_refine(ds, nb, s, lo, hi, steps=10, step0=0.01, rows=rows)
              for s in starts]
    multi = oracle.crs_refine_multi(ds, nb, starts, lo, hi, steps=10, step0=0.01, rows=rows)
    np.testing.assert_array_equal(multi.S, np.maximum(single[0].S, single[1].S))
    pick = np.where(single[1].S > single[0].S, 1, 0)
    for r in range(3):
        np.testing.assert_array_equal(multi.theta[r], single[pick[r]].theta[r])
    assert multi.S[1] > 0.999          # the start next to the exact operator wins


def test_pragmatic_crs_recovers_exact_plane():
    """Exactly sampled dipping plane (A = 2^-6, B = 0, C = 2^-20) stored as 7 CMP gathers:
    the central CMP's traces give C, the 7 zero-offset traces give A and B, and the combined
    operator has S = 1 over the full aperture."""
    ds, (At, Bt, Ct) = _exact_plane()
    _, sizes = np.unique(ds["m"], return_counts=True)        # traces are grouped by CMP
    ds = dataset([ds["traces"][ds["trace_off"][i]:ds["trace_off"][i + 1]]
                  for i in range(len(ds["h"]))], ds["h"], 1.0 / 256, m=ds["m"],
                 gather_sizes=list(sizes))
    A = At * np.array([0.5, 1.0, 1.5]); B = np.array([-2.0 ** -10, 0.0, 2.0 ** -10])
    C = Ct * np.array([0.8, 1.0, 1.2])
    assert len(oracle.offset_limited(ds, oracle.aperture(ds, [3], 3.0), 0.0)[1]) == 7
    r = oracle.crs_pragmatic(ds, [3], 3.0, 0.0, A, B, C, c_zo=C[0])
    np.testing.assert_array_equal(r.theta[260], [At, 0.0, Ct])
    assert r.S[260] == pytest.approx(1.0, abs=1e-12)
    assert r.gap_cmp[260] > 1e-3 and r.gap_zo[260] > 1e-3


# --- t0-window semblance (reading c18) --------------------------------------------------

def _t0win_brute(ds, C, w, g, n):
    """The reading c18 definition written out in plain Python for one (gather, row)."""
    hw = w // 2
    t0s = [(n + j) for j in range(-hw, hw + 1)]
    nrow = int(ds["out_off"][g + 1] - ds["out_off"][g])
    dt = float(ds["dt"][g])
    out = []
    for Cc in C:
        num = den = 0.0
        for n2 in t0s:
            if n2 < 0 or n2 >= nrow:
                continue
            s = e = 0.0
            M = 0
            for i in range(int(ds["gather_off"][g]), int(ds["gather_off"][g + 1])):
                f = ds["traces"][ds["trace_off"][i]:ds["trace_off"][i + 1]]
                u = math.sqrt((n2 * dt) ** 2 + float(Cc) * float(ds["h"][i]) ** 2) / dt
                k = math.floor(u)
                if k < 0 or k + 1 > len(f) - 1:
                    continue
                v = float(f[k]) + (u - k) * (float(f[k + 1]) - float(f[k]))
                s += v
                e += v * v
                M += 1
            num += s * s
            den += M * e
        out.append(num / den if den > 0 else 0.0)
    return np.array(out)


def test_t0win_brute_force_tiny():
    rng = np.random.default_rng(21)
    traces = [rng.normal(size=40) for _ in range(5)]
    ds = dataset(traces, [0.0, 10.0, 35.0, 60.0, 90.0], 0.004, gather_sizes=[3, 2])
    C = np.float32([0.0, 3e-7, 1.2e-6, 4e-6])
    r = oracle.cmp_semblance(ds, C, w=5, t0_window=True)
    for row in (0, 1, 7, 20, 38, 39, 40, 45, 79):
        g = 0 if row < 40 else 1
        np.testing.assert_allclose(r.S[row], _t0win_brute(ds, C, 5, g, row - 40 * g),
                                   rtol=1e-12, atol=1e-15)


def test_t0win_equals_paper_window_at_zero_moveout():
    """At C = 0 every traveltime is the output time itself (x = 0), so on rows whose whole
    window lies inside every trace the two windows read the same samples: equal S."""
    rng = np.random.default_rng(22)
    ds = dataset([rng.normal(size=120) for _ in range(6)], np.linspace(0, 500, 6), 0.004)
    a = oracle.cmp_semblance(ds, [0.0], w=7)
    b = oracle.cmp_semblance(ds, [0.0], w=7, t0_window=True)
    rows = np.arange(3, 116)                  # k - 3 >= 0 and k + 4 <= 119
    np.testing.assert_allclose(b.S[rows, 0], a.S[rows, 0], rtol=1e-12, atol=1e-15)


def test_t0win_invariants():
    rng = np.random.default_rng(23)
    C = np.float32(np.linspace(0, 2e-6, 9))
    ds = dataset([np.full(200, 1.7) for _ in range(4)], [0, 100, 300, 700], 0.004)
    r = oracle.cmp_semblance(ds, C, w=11, t0_window=True)
    live = r.N > 0
    np.testing.assert_allclose(r.S[live], 1.0, rtol=0, atol=1e-14)     # constant traces
    one = dataset([rng.normal(size=150)], [250.0], 0.004)
    r1 = oracle.cmp_semblance(one, C, w=9, t0_window=True)
    np.testing.assert_allclose(r1.S[r1.N > 0], 1.0, rtol=0, atol=1e-14)  # a single trace
    noisy = dataset([rng.normal(size=300) for _ in range(8)], np.linspace(0, 1400, 8), 0.004)
    r2 = oracle.cmp_semblance(noisy, C, w=11, t0_window=True)
    assert np.all(r2.S >= 0) and np.all(r2.S <= 1 + 1e-12)              # Cauchy-Schwarz
    zero = dataset([np.zeros(100) for _ in range(3)], [0, 50, 90], 0.004)
    assert np.all(oracle.cmp_semblance(zero, C, t0_window=True).S == 0)


def test_crs_t0win_reduces_to_cmp_t0win():
    """dm = 0 (each gather its own aperture) and A = B = 0: the CRS t0-window search is the
    CMP one, bit for bit (the same FP64 operations)."""
    rng = np.random.default_rng(31)
    ds = dataset([rng.normal(size=180) for _ in range(10)], np.tile(np.linspace(0, 900, 5), 2),
                 0.004, gather_sizes=[5, 5])
    C = np.float32(np.linspace(0, 2e-6, 7))
    a = oracle.cmp_semblance(ds, C, w=9, t0_window=True)
    b = oracle.crs_semblance(ds, oracle.cmp_as_crs(ds), [0.0], [0.0], C, w=9, want_cube=True,
                             t0_window=True)
    np.testing.assert_array_equal(a.S, b.S)
    np.testing.assert_array_equal(a.best_idx, b.best_idx)
    np.testing.assert_array_equal(a.stack, b.stack)


def test_crs_t0win_constant_traces():
    ds = dataset([np.full(150, -0.8) for _ in range(9)], np.tile([0, 300, 600], 3), 0.004,
                 m=np.repeat([0.0, 12.5, 25.0], 3), gather_sizes=[3, 3, 3])
    nb = oracle.aperture(ds, [1], 12.5)
    r = oracle.crs_semblance(ds, nb, [-1e-4, 0, 1e-4], [0.0, 1e-7], [0.0, 1e-6], w=5,
                             want_cube=True, t0_window=True)
    live = r.N > 0
    assert live.mean() > 0.5
    np.testing.assert_allclose(r.S[live], 1.0, rtol=0, atol=1e-14)


def test_invalid_arguments():
    ds = dataset([np.zeros(50)], [0.0], 0.004)
    with pytest.raises(ValueError):
        oracle.cmp_semblance(ds, [1e-6], w=4)
    with pytest.raises(ValueError):
        oracle.cmp_semblance(ds, [1e-6], w=0)


# --- admissible ranges where FP32 may decide a trace's participation either way (c5) ---

def _window_S(windows, w):
    """Eq. 1 (with 1/N) and Algorithm 1's stack from the traces' interpolated windows."""
    if not windows:
        return 0.0, 0.0
    num = [sum(v[j] for v in windows) for j in range(w)]
    den = sum(x * x for v in windows for x in v)
    N = len(windows)
    S = sum(a * a for a in num) / (N * den) if den > 0 else 0.0
    return S, sum(sum(v) for v in windows) / (N * w)


def test_admissible_range_at_mask_edges_bruteforce():
    """Row 3 (dt = 1/256 s, C = 2^-20): trace 0 (h = 16 m, 8 samples) meets u = 5 exactly,
    where w = 5 needs k + 3 <= 7, so it is out in exact arithmetic but in at k = 4, x = 1 for
    an FP32 u a hair below 5.  Row 0: trace 1 (h = 8 m) meets u = 2 = hw exactly, in at
    k = 2, x = 0, but out for u a hair below 2.  The oracle's range of S, stack and N must be
    the min / max over exactly those two outcomes (computed here by brute force with
    numpy.interp); entries with no trace on an edge have a range of zero width."""
    rng = np.random.default_rng(77)
    dt, w, hw = 1.0 / 256.0, 5, 2
    traces = [rng.standard_normal(8), rng.standard_normal(20), rng.standard_normal(20),
              rng.standard_normal(20)]
    h = [16.0, 8.0, 0.0, 12.0]
    ds = dataset(traces, h, dt, out_ns=[10])
    C = np.float32([2.0 ** -20, 1.5 * 2.0 ** -20])
    r = oracle.cmp_semblance(ds, C, w=w)
    f = [np.asarray(t, np.float32).astype(np.float64) for t in traces]

    def win(i, u):
        return [float(np.interp(u + j, np.arange(len(f[i])), f[i])) for j in range(-hw, hw + 1)]

    def inside(i, u):
        k = np.floor(u)
        return k - hw >= 0 and k + hw + 1 <= len(f[i]) - 1

    for n, edge_tr in ((3, 0), (0, 1)):
        us = [np.sqrt(n * n + 2.0 ** -20 * hh * hh / dt ** 2) for hh in h]
        assert us[edge_tr] == (5.0 if n == 3 else 2.0)
        base = [win(i, us[i]) for i in range(4) if i != edge_tr and inside(i, us[i])]
        outcomes = [_window_S(base, w), _window_S(base + [win(edge_tr, us[edge_tr])], w)]
        Ss = [o[0] for o in outcomes]
        sts = [o[1] for o in outcomes]
        assert r.edge[n, 0] == 1
        assert r.S_lo[n, 0] == pytest.approx(min(Ss), abs=1e-14)
        assert r.S_hi[n, 0] == pytest.approx(max(Ss), abs=1e-14)
        assert r.st_lo[n, 0] == pytest.approx(min(sts), abs=1e-14)
        assert r.st_hi[n, 0] == pytest.approx(max(sts), abs=1e-14)
        assert (r.N_lo[n, 0], r.N_hi[n, 0]) == (len(base), len(base) + 1)
        # the nominal (exact-arithmetic) result is the outcome u itself gives
        nominal = 1 if inside(edge_tr, us[edge_tr]) else 0
        assert r.S[n, 0] == pytest.approx(Ss[nominal], abs=1e-14)
        assert abs(max(Ss) - min(Ss)) > 1e-3            # the edge matters here
    plain = r.edge == 0
    assert plain.sum() >= 15
    np.testing.assert_array_equal(r.S_lo[plain], r.S[plain])
    np.testing.assert_array_equal(r.S_hi[plain], r.S[plain])
    np.testing.assert_array_equal(r.st_lo[plain], r.stack_at[plain])
    np.testing.assert_array_equal(r.stack_at[np.arange(10), r.best_idx], r.stack)


def test_admissible_range_t0win_bruteforce():
    """t0-window semblance (w = 3) at row 3: at t0' = 3 dt trace 0 (6 samples, h = 16 m)
    meets u = 5 exactly, out in exact arithmetic (k + 1 = 6 > 5) but in at k = 4, x = 1 for
    u a hair below 5; its other window rows are not on an edge.  The range is the min / max
    of the two outcomes (brute force)."""
    rng = np.random.default_rng(78)
    dt, w = 1.0 / 256.0, 3
    traces = [rng.standard_normal(6), rng.standard_normal(20), rng.standard_normal(20)]
    h = [16.0, 0.0, 10.0]
    ds = dataset(traces, h, dt, out_ns=[8])
    C = np.float32([2.0 ** -20])
    r = oracle.cmp_semblance(ds, C, w=w, t0_window=True)
    f = [np.asarray(t, np.float32).astype(np.float64) for t in traces]
    n = 3

    def S_of(force_in):
        s, e, M = [], [], []
        for n2 in (n - 1, n, n + 1):
            vals = []
            for i in range(3):
                u = np.sqrt(n2 * n2 + 2.0 ** -20 * h[i] ** 2 / dt ** 2)
                ok = np.floor(u) >= 0 and np.floor(u) + 1 <= len(f[i]) - 1
                if i == 0 and n2 == n:
                    assert u == 5.0 and not ok
                    ok = force_in
                if ok:
                    vals.append(float(np.interp(min(u, len(f[i]) - 1), np.arange(len(f[i])), f[i])))
            s.append(sum(vals)); e.append(sum(v * v for v in vals)); M.append(len(vals))
        den = sum(m * x for m, x in zip(M, e))
        return sum(x * x for x in s) / den, s[1] / M[1]

    outs = [S_of(False), S_of(True)]
    assert r.edge[n, 0] == 1
    assert r.S_lo[n, 0] == pytest.approx(min(o[0] for o in outs), abs=1e-14)
    assert r.S_hi[n, 0] == pytest.approx(max(o[0] for o in outs), abs=1e-14)
    assert r.st_lo[n, 0] == pytest.approx(min(o[1] for o in outs), abs=1e-14)
    assert r.st_hi[n, 0] == pytest.approx(max(o[1] for o in outs), abs=1e-14)
    assert r.S[n, 0] == pytest.approx(outs[0][0], abs=1e-14)
