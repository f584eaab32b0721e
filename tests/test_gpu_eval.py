"""Per-row operator evaluation on the GPU (stack, adjoint, refinement, autograd) against
the FP64 oracle."""
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


def _ranges():
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    return np.array([alo, blo, clo]), np.array([ahi, bhi, chi])


@pytest.fixture(scope="module")
def line(seis):
    ds = synth.crs_line(20, 12, 500, 0.004, 0.0, 1800.0, 3, 2, 2.0, seed=61)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, np.arange(4, 16), 50.0)
    ap.oracle_nb = oracle.aperture(ds, np.arange(4, 16), 50.0)   # the oracle's own lists
    return ds, g, ap


def _random_theta(rows, seed, shrink=0.6):
    lo, hi = _ranges()
    rng = np.random.default_rng(seed)
    mid, half = (lo + hi) / 2, (hi - lo) / 2 * shrink
    th = mid + half * rng.uniform(-1, 1, (rows, 3))
    th[:, 2] = rng.uniform(lo[2], hi[2], rows)
    return th.astype(np.float32)


def test_stack_cmp_matches_oracle(seis):
    ds = synth.cmp_line(5, 14, 400, 0.004, 0.0, 1600.0, 3, 2.0, seed=71)
    g = seis.to_device(ds)
    rows = int(ds["out_off"][-1])
    rng = np.random.default_rng(3)
    C = np.float32(4.0 / rng.uniform(1400, 4500, rows) ** 2)
    out = seis.stack(g, None, torch.from_numpy(C).cuda(), w=11)
    torch.cuda.synchronize()
    seis.device_status()
    th = np.stack([np.zeros(rows), np.zeros(rows), C.astype(np.float64)], 1)
    ref = oracle.crs_eval(ds, oracle.cmp_as_crs(ds), th)
    parity.check_eval(out["S"].cpu().numpy(), out["stack"].cpu().numpy(),
                      out["N"].cpu().numpy(), ref, "stack-cmp")


def test_stack_matches_search_pick(seis):
    """stack() at the search's picked C reproduces the search's stack and best S bit for bit."""
    ds = synth.cmp_line(3, 16, 300, 0.004, 0.0, 1500.0, 3, 2.0, seed=72)
    g = seis.to_device(ds)
    C = torch.from_numpy(oracle.velocity_grid(1400, 4500, 61).astype(np.float32)).cuda()
    srch = seis.cmp_semblance(g, C, w=11)
    out = seis.stack(g, None, srch["best_C"], w=11)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["stack"].cpu().numpy(), srch["stack"].cpu().numpy())
    np.testing.assert_array_equal(out["S"].cpu().numpy(), srch["best_S"].cpu().numpy())


def test_stack_crs_matches_oracle(seis, line):
    ds, g, ap = line
    th = _random_theta(ap.rows, 5)
    out = seis.stack(g, ap, torch.from_numpy(th).cuda(), w=11)
    torch.cuda.synchronize()
    seis.device_status()
    ref = oracle.crs_eval(ds, ap.oracle_nb, th.astype(np.float64))
    # every row: N, S and the stack inside the oracle's admissible ranges (a row where FP32
    # may decide a trace's participation either way has the range of both outcomes)
    rep = parity.check_eval(out["S"].cpu().numpy(), out["stack"].cpu().numpy(),
                            out["N"].cpu().numpy(), ref, "stack-crs")
    assert rep["flagged"] < 0.05


def test_adjoint_matches_oracle_gradient(seis, line):
    ds, g, ap = line
    th = _random_theta(ap.rows, 6)
    S, grad, st = seis.crs_semblance_grad(g, ap, torch.from_numpy(th).cuda(), w=11)
    torch.cuda.synchronize()
    seis.device_status()
    ref = oracle.crs_eval(ds, ap.oracle_nb, th.astype(np.float64))
    G = grad.cpu().numpy().astype(np.float64)
    # rows with a trace within FP32 reach of a sample point are skipped: the derivative is
    # defined almost everywhere and FP32 may land on the other side of the knot
    assert ref.knot.mean() <= 0.3, ref.knot.mean()
    live = (ref.S > 0.05) & ~ref.knot
    for a, name in enumerate("ABC"):
        e = G[live, a] - ref.grad[live, a]
        rel = np.linalg.norm(e) / np.linalg.norm(ref.grad[live, a])
        med = np.median(np.abs(e) / (np.abs(ref.grad[live, a]) + 1e-12))
        print(f"[parity] grad d/d{name}: rel L2 {rel:.2e}, median row rel {med:.2e}")
        assert rel <= 1e-3 and med <= 1e-3
    assert np.abs(S.cpu().numpy() - ref.S)[~ref.knot].max() <= parity.S_TOL


def test_autograd_function_uses_adjoint(seis, line):
    ds, g, ap = line
    th = torch.from_numpy(_random_theta(ap.rows, 7)).cuda().requires_grad_(True)
    S = seis.crs_semblance_at(th, g, ap, 11)
    wts = torch.linspace(0.5, 1.5, ap.rows, device="cuda")
    (S * wts).sum().backward()
    S2, dS, _ = seis.crs_semblance_grad(g, ap, th.detach(), w=11)
    torch.testing.assert_close(S.detach(), S2, rtol=0, atol=0)
    torch.testing.assert_close(th.grad, wts[:, None] * dS, rtol=0, atol=0)


@pytest.fixture(scope="module")
def coarse_starts(line):
    """The oracle's coarse 7x7x11 search on the test line and its 4 best candidates per
    row: the starting operators both sides refine from."""
    ds, g, ap = line
    lo, hi = _ranges()
    A = np.float32(np.linspace(lo[0], hi[0], 7)); B = np.float32(np.linspace(lo[1], hi[1], 7))
    C = np.float32(np.linspace(lo[2], hi[2], 11))
    ref = oracle.crs_semblance(ds, ap.oracle_nb, A, B, C, want_cube=True)
    return ref, oracle.top_starts(ref.S, A, B, C, 4)


def test_refine_monotone_and_consistent(seis, line, coarse_starts):
    ds, g, ap = line
    lo, hi = _ranges()
    coarse, starts = coarse_starts
    th0 = torch.from_numpy(starts[0].astype(np.float32)).cuda()
    S0 = seis.stack(g, ap, th0, w=11)["S"].cpu().numpy()
    r = seis.crs_refine(g, ap, th0, lo, hi, steps=20, step0=0.05, w=11)
    torch.cuda.synchronize()
    seis.device_status()
    S1 = r["S"].cpu().numpy()
    th1 = r["theta"].cpu().numpy()
    assert np.all(S1 >= S0 - 1e-6)
    assert np.all(th1 >= np.float32(lo) - 1e-12) and np.all(th1 <= np.float32(hi) + 1e-12)
    # the reported S is that of the reported operator (the evaluation kernel at it)
    S_at = seis.stack(g, ap, r["theta"], w=11)["S"].cpu().numpy()
    np.testing.assert_allclose(S1, S_at, rtol=0, atol=1e-6)
    # against the oracle's own refinement from the same start
    ref = oracle.crs_refine(ds, ap.oracle_nb, starts[0], lo, hi, steps=20, step0=0.05)
    close = np.abs(S1 - ref.S) <= 1e-3
    print(f"[parity] refine: gain {np.mean(S1 - S0):.4f}, |S_gpu - S_oracle| <= 1e-3 on "
          f"{close.mean():.3f} of rows, mean diff {np.mean(S1 - ref.S):+.2e}")
    assert close.mean() >= 0.9


@pytest.mark.parametrize("steps", [1, 2])
def test_refine_steps_elementwise(seis, line, coarse_starts, steps):
    """One and two refinement trials from the oracle's best coarse candidates, compared with
    the oracle's trajectory element by element.  The trial direction is d = H g, so an FP32
    gradient with relative error e moves the trial by about 2 e |d|; the GPU's gradient
    error is measured at the start and at the oracle's trial points (the adjoint entry point
    runs the refinement's evaluation kernel), and each row's operator must land within the
    first-order bound that these errors give (BFGS step: the errors of g1 and of
    y = g0 - g1 relative to |y|).  Rows are compared where the start and every trial are
    knot-free (the gradient is defined in both precisions) and every accept decision is
    clear (|S' - S| > 5e-5)."""
    ds, g, ap = line
    lo, hi = _ranges()
    span = hi - lo
    nb = ap.oracle_nb
    _, starts = coarse_starts
    th0 = starts[0].astype(np.float32)
    r = seis.crs_refine(g, ap, torch.from_numpy(th0).cuda(), lo, hi, steps=steps, step0=0.05,
                        w=11)
    torch.cuda.synchronize()
    seis.device_status()
    ref = oracle.crs_refine(ds, nb, th0.astype(np.float64), lo, hi, steps=steps, step0=0.05)

    def gpu_grad(th):
        _, G, _ = seis.crs_semblance_grad(g, ap, torch.from_numpy(th.astype(np.float32)).cuda(),
                                          w=11)
        return G.cpu().numpy().astype(np.float64) * span

    pts = [th0.astype(np.float64)] + [np.nan_to_num(ref.traj[:, it, :3]) for it in range(steps)]
    ev = [oracle.crs_eval(ds, nb, p) for p in pts]
    gz = [e.grad * span for e in ev]                               # dS/dz, oracle
    err = [np.linalg.norm(gpu_grad(p) - q, axis=1) for p, q in zip(pts, gz)]
    nrm = [np.linalg.norm(q, axis=1) for q in gz]
    robust = (ev[0].S > 0.02) & ~ev[0].knot & (nrm[0] > 0)
    S_prev = ev[0].S.copy()
    for it in range(steps):
        tr = ref.traj[:, it]
        robust &= ~np.isnan(tr[:, 3]) & ~ev[it + 1].knot & (np.abs(tr[:, 3] - S_prev) > 5e-5)
        S_prev = np.where(tr[:, 4] == 1.0, tr[:, 3], S_prev)
    z = lambda th: (th - lo) / span
    rel0 = err[0] / np.maximum(nrm[0], 1e-30)
    tol1 = 1e-6 + 2.0 * 0.05 * rel0                                # |d1| = step0 = 0.05
    acc1 = ref.traj[:, 0, 4] == 1.0
    if steps == 1:
        tol = np.where(acc1, tol1, 1e-6)
    else:
        acc2 = ref.traj[:, 1, 4] == 1.0
        sv = z(ref.traj[:, 0, :3]) - z(pts[0])
        yv = gz[0] - gz[1]
        s_n, y_n = np.linalg.norm(sv, axis=1), np.linalg.norm(yv, axis=1)
        kappa = s_n * y_n / np.maximum(np.abs(np.sum(sv * yv, axis=1)), 1e-300)
        ey = (err[0] + err[1]) / np.maximum(y_n, 1e-30)
        rel1 = err[1] / np.maximum(nrm[1], 1e-30)
        # d2 = H1 g1 with H1 = V'H0V + rho s s', V = I - rho y s', H0 = (0.05/|g0|) I: the
        # sizes of its two terms, times the relative errors of g0 (H0's scale), g1, and y
        # (which enters through rho = 1/(s.y), amplified by kappa = |s||y|/|s.y|)
        T = nrm[1] * (0.05 / np.maximum(nrm[0], 1e-30) * (1.0 + kappa) ** 2
                      + kappa * s_n / np.maximum(y_n, 1e-30))
        tol2_acc = tol1 * (1.0 + 2.0 * kappa) + T * (rel0 + rel1 + 2.0 * kappa * ey)
        tol2_rej = 1e-6 + 0.5 * (tol1 - 1e-6)                              # halved first trial
        tol_trial2 = np.where(acc1, tol2_acc, tol2_rej)
        tol = np.where(acc2, tol_trial2, np.where(acc1, tol1, 1e-6))
    th_g = r["theta"].cpu().numpy().astype(np.float64)
    dz = np.linalg.norm(z(th_g) - z(ref.theta), axis=1)
    # the GPU's final operator is knot-free too, so its S and gradient are continuous there
    eg = oracle.crs_eval(ds, nb, th_g)
    robust &= ~eg.knot
    sel = robust
    S_g = r["S"].cpu().numpy().astype(np.float64)
    G_g = r["grad"].cpu().numpy().astype(np.float64) * span
    dS = np.abs(S_g - ref.S)
    dG = np.linalg.norm(G_g - eg.grad * span, axis=1)
    nG = np.linalg.norm(eg.grad * span, axis=1)
    print(f"[parity] refine {steps} step(s): {sel.sum()} of {len(sel)} rows compared; "
          f"|dz| max {dz[sel].max():.2e}, 99th pct {np.percentile(dz[sel], 99):.2e}, "
          f"max |dz|/bound {np.max(dz[sel] / tol[sel]):.2f}; max |dS| {dS[sel].max():.2e}; "
          f"grad at the GPU's operator: median rel {np.median(dG[sel] / nG[sel]):.2e}")
    assert sel.mean() > 0.3
    bad = sel & (dz > tol)
    assert not bad.any(), (f"{bad.sum()} rows beyond the FP32 bound, e.g. row "
                           f"{np.nonzero(bad)[0][0]}: |dz| {dz[bad][0]:.2e} > {tol[bad][0]:.2e}")
    # S: the oracle's S at its own point, plus the first-order change over |dz|
    assert np.all(dS[sel] <= parity.S_TOL + nrm[-1][sel] * dz[sel] * 2.0 + 1e-6)
    # the reported S and gradient are the evaluation at the reported operator: against the
    # oracle there (relative 1e-3 of the gradient, with an FP32 floor)
    assert np.all(np.abs(S_g - eg.S)[sel] <= parity.S_TOL)
    # the gradient is the evaluation kernel's at the reported operator, bit for bit, and that
    # kernel's gradient matches the oracle's there as the adjoint test requires
    np.testing.assert_array_equal(G_g, gpu_grad(th_g.astype(np.float32)))
    rel = np.linalg.norm((G_g - eg.grad * span)[sel]) / np.linalg.norm((eg.grad * span)[sel])
    assert rel <= 1e-3 and np.median(dG[sel] / nG[sel]) <= 1e-3, rel


def test_top_starts_exact(seis):
    """Selection of refinement starts: integer work on a cube full of ties, bit-exact."""
    rows, (nA, nB, nC) = 333, (5, 3, 7)
    cube = synth.score_cube(rows, nA * nB * nC, levels=5, seed=17)
    A = np.float32(np.linspace(-1, 1, nA)); B = np.float32(np.linspace(2, 3, nB))
    C = np.float32(np.linspace(5, 9, nC))
    t = lambda a: torch.from_numpy(a).cuda()
    for k in (1, 6, nA * nB * nC):
        got = seis.crs_top_starts(t(cube), t(A), t(B), t(C), k).cpu().numpy()
        want = oracle.top_starts(cube, A, B, C, k).astype(np.float32)
        np.testing.assert_array_equal(got, want)
    with pytest.raises(seis.SeisError):
        seis.crs_top_starts(t(cube), t(A), t(B), t(C), nA * nB * nC + 1)


def test_local_max_starts_exact(seis):
    """Starts at the cube's local maxima: integer work on cubes full of ties, bit-exact
    against the oracle's definition, for several grid shapes (one axis of length 1 too)."""
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for rows, (nA, nB, nC), k in [(333, (5, 3, 7), 6), (100, (7, 7, 11), 16), (64, (1, 1, 41), 5),
                                  (50, (4, 1, 3), 12)]:
        cube = synth.score_cube(rows, nA * nB * nC, levels=4, seed=nA + nC)
        A = np.float32(np.linspace(-1, 1, nA)); B = np.float32(np.linspace(2, 3, nB))
        C = np.float32(np.linspace(5, 9, nC))
        got = seis.crs_top_starts(t(cube), t(A), t(B), t(C), k, local_max=True).cpu().numpy()
        want = oracle.local_max_starts(cube, A, B, C, k).astype(np.float32)
        np.testing.assert_array_equal(got, want)
    with pytest.raises(seis.SeisError):
        seis.crs_top_starts(t(cube), t(A), t(B), t(C), nA * nB * nC + 1, local_max=True)


def test_refine_multi(seis, line, coarse_starts):
    ds, g, ap = line
    lo, hi = _ranges()
    _, starts = coarse_starts
    st = torch.from_numpy(starts.astype(np.float32)).cuda()
    multi = seis.crs_refine_multi(g, ap, st, lo, hi, steps=20, step0=0.05, w=11)
    single = seis.crs_refine(g, ap, st[0], lo, hi, steps=20, step0=0.05, w=11)
    torch.cuda.synchronize()
    seis.device_status()
    Sm = multi["S"].cpu().numpy()
    Ss = single["S"].cpu().numpy()
    # start 0 runs the same arithmetic as the single refinement, so the best of all starts
    # is never below it
    assert np.all(Sm >= Ss)
    thm = multi["theta"].cpu().numpy()
    assert np.all(thm >= np.float32(lo) - 1e-12) and np.all(thm <= np.float32(hi) + 1e-12)
    ref = oracle.crs_refine_multi(ds, ap.oracle_nb, starts, lo, hi, steps=20, step0=0.05)
    close = np.abs(Sm - ref.S) <= 1e-3
    print(f"[parity] refine multi (4 starts): gain over one start {np.mean(Sm - Ss):.4f}, "
          f"|S_gpu - S_oracle| <= 1e-3 on {close.mean():.3f} of rows")
    assert close.mean() >= 0.9


@pytest.mark.parametrize("nstart", [2, 3])
def test_refine_multi_pairs_equal_single_refinements_bitwise(seis, line, coarse_starts, nstart):
    """crs_refine_multi refines the starts two at a time in one paired evaluation kernel (an
    odd last start alone); its result equals the best of separate crs_refine runs, chosen
    with the earlier start on ties, bit for bit."""
    ds, g, ap = line
    lo, hi = _ranges()
    _, starts = coarse_starts
    st = torch.from_numpy(starts[:nstart].astype(np.float32)).cuda()
    multi = seis.crs_refine_multi(g, ap, st, lo, hi, steps=6, step0=0.05, w=11)
    single = [seis.crs_refine(g, ap, st[k], lo, hi, steps=6, step0=0.05, w=11)
              for k in range(nstart)]
    torch.cuda.synchronize()
    seis.device_status()
    best = {k: v.clone() for k, v in single[0].items()}
    for r in single[1:]:
        better = r["S"] > best["S"]
        for k in best:
            best[k][better] = r[k][better]
    for k in ("theta", "S", "grad", "stack"):
        assert torch.equal(multi[k], best[k]), k


def test_refine_workload_sample(seis):
    """The refinement workload (aperture +-8 CMPs = 816 traces, 2000 samples) on two central
    CMPs: both sides refine from the oracle's 4 best 7 x 7 x 11 candidates of every row; the
    oracle's multi-start refinement checks every 40th row."""
    ds = synth.workload_crs_refine()
    central = ds["central"][[0, 300]]
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, central, ds["apm"])
    nb = oracle.aperture(ds, central, ds["apm"])
    assert int(ap.nbr_off[1] - ap.nbr_off[0]) == 816
    lo, hi = _ranges()
    A = np.float32(np.linspace(lo[0], hi[0], 7)); B = np.float32(np.linspace(lo[1], hi[1], 7))
    C = np.float32(np.linspace(lo[2], hi[2], 11))
    coarse = oracle.crs_semblance(ds, nb, A, B, C, want_cube=True)
    starts = oracle.top_starts(coarse.S, A, B, C, 4)
    st = torch.from_numpy(starts.astype(np.float32)).cuda()
    multi = seis.crs_refine_multi(g, ap, st, lo, hi, steps=20, step0=0.05, w=11)
    torch.cuda.synchronize()
    seis.device_status()
    Sm = multi["S"].cpu().numpy()
    S0 = seis.stack(g, ap, st[0], w=11)["S"].cpu().numpy()
    assert np.all(Sm >= S0 - 1e-6)                 # never below the best coarse start
    rows = np.arange(0, ap.rows, 40)
    ref = oracle.crs_refine_multi(ds, nb, starts[:, rows], lo, hi, steps=20, step0=0.05,
                                  rows=rows)
    close = np.abs(Sm[rows] - ref.S) <= 1e-3
    print(f"[parity] refine workload: |S_gpu - S_oracle| <= 1e-3 on {close.mean():.3f} of "
          f"{len(rows)} rows")
    assert close.mean() >= 0.9
