"""CRS aperture build and CRS semblance search on the GPU (through the C ABI) against
the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1907_11678_gb300 import synth
from tests import parity
from tests.dsutil import dataset, pythagorean_offsets, spike_wavelet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def seis():
    from paper_1907_11678_gb300 import build, seis as s
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return s


def _grids(nA, nB, nC):
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    return (oracle.linear_grid(alo, ahi, nA).astype(np.float32),
            oracle.linear_grid(blo, bhi, nB).astype(np.float32),
            oracle.linear_grid(clo, chi, nC).astype(np.float32))


def _nb_of(ap):
    return (ap.nbr_off.cpu().numpy(), ap.nbr_trace.cpu().numpy()[:int(ap.nbr_off[-1])],
            ap.m_c.cpu().numpy(), ap.out_off.cpu().numpy(), ap.dt.cpu().numpy())


def _run(seis, g, ap, A, B, C, w=11, cube=True):
    t = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    out = seis.crs_semblance(g, ap, t(A), t(B), t(C), w=w, want_cube=cube)
    torch.cuda.synchronize()
    seis.device_status()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_aperture_matches_oracle(seis):
    ds = synth.crs_line(30, 4, 200, 0.004, 0.0, 500.0, 1, 0, None, seed=2)
    central = np.array([0, 7, 15, 29], np.int32)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, central, 37.5)
    off, tr, mc = oracle.neighbours(ds, central, 37.5)
    got = _nb_of(ap)
    np.testing.assert_array_equal(got[0], off)
    np.testing.assert_array_equal(got[1], tr)
    np.testing.assert_array_equal(got[2], mc)
    np.testing.assert_array_equal(got[3], np.arange(5) * 200)
    np.testing.assert_array_equal(got[4], np.float32([0.004] * 4))
    assert ap.max_rows == 200 and ap.rows == 800


def test_aperture_rejects_bad_central(seis):
    ds = synth.crs_line(5, 4, 100, 0.004, 0.0, 500.0, 1, 0, None, seed=2)
    g = seis.to_device(ds)
    with pytest.raises(seis.SeisError):
        seis.crs_aperture(g, [1, 9], 20.0)


def test_crs_small_full_cube(seis):
    ds = synth.crs_line(9, 12, 300, 0.004, 0.0, 1500.0, 2, 1, 2.0, seed=41)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, [3, 4, 5], 30.0)
    nb = oracle.aperture(ds, [3, 4, 5], 30.0)
    A, B, C = _grids(5, 3, 7)
    got = _run(seis, g, ap, A, B, C)
    ref = oracle.crs_semblance(ds, nb, A, B, C, want_cube=True)
    parity.check_cube(got["S"], ref, "crs-small")
    parity.check_picks(got["best_idx"], got["best_S"], got["stack"], ref, "crs-small")
    ia, rem = np.divmod(got["best_idx"], 3 * 7)
    ib, ic = np.divmod(rem, 7)
    np.testing.assert_array_equal(got["best_ABC"], np.stack([A[ia], B[ib], C[ic]], 1))


@pytest.mark.parametrize("w", [1, 5, 15])
def test_crs_windows_and_ragged(seis, w):
    """Uneven aperture sizes (line ends), odd candidate counts, several windows."""
    ds = synth.crs_line(7, 5, 170, 0.004, 0.0, 1200.0, 2, 1, 1.5, seed=50 + w)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, [0, 3, 6], 25.0)
    nb = oracle.aperture(ds, [0, 3, 6], 25.0)
    A, B, C = _grids(3, 2, 9)
    got = _run(seis, g, ap, A, B, C, w=w)
    ref = oracle.crs_semblance(ds, nb, A, B, C, w=w, want_cube=True)
    parity.check_cube(got["S"], ref, f"crs-w{w}")
    parity.check_picks(got["best_idx"], got["best_S"], got["stack"], ref, f"crs-w{w}")


def test_crs_exact_dipping_plane(seis):
    n0, ns, dt = 260, 700, 1.0 / 256.0
    traces, h, m = [], [], []
    for dm in range(-3, 4):
        p = n0 + 4 * dm
        for a, mm in [(0, p)] + pythagorean_offsets(p, 90)[:6]:
            traces.append(spike_wavelet(ns, mm, 2.5)); h.append(16.0 * a); m.append(100.0 + dm)
    ds = dataset(traces, h, dt, m=m, gather_sizes=[1] * len(traces))
    # the central gather is the first dm = 0 trace
    cen = [i for i, mm in enumerate(m) if mm == 100.0][0]
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, [cen], 3.0)
    assert int(ap.nbr_off[-1]) == len(traces)
    At, Ct = 2.0 ** -6, 2.0 ** -20
    A = np.float32(At * np.array([0.5, 1.0, 1.5]))
    B = np.float32([-2.0 ** -10, 0.0, 2.0 ** -10])
    C = np.float32(Ct * np.array([0.8, 1.0, 1.2]))
    got = _run(seis, g, ap, A, B, C)
    true = (1 * 3 + 1) * 3 + 1
    assert got["S"][n0, true] == pytest.approx(1.0, abs=1e-5)
    assert got["best_idx"][n0] == true


def test_crs_zero_dm_equals_cmp_bitwise(seis):
    """With every gather as its own aperture (dm = 0) and A = B = 0, the CRS kernel
    reproduces the CMP kernel bit for bit (the dm = 0 reduction of the CRS operator)."""
    ds = synth.cmp_line(4, 16, 400, 0.004, 0.0, 2000.0, 3, 1.0, seed=77)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, np.arange(4), 0.0)
    C = oracle.velocity_grid(1400.0, 4500.0, 45).astype(np.float32)
    crs = _run(seis, g, ap, [0.0], [0.0], C)
    cmp = seis.cmp_semblance(g, torch.from_numpy(C).cuda(), w=11, want_cube=True)
    np.testing.assert_array_equal(crs["S"], cmp["S"].cpu().numpy())
    np.testing.assert_array_equal(crs["best_idx"], cmp["best_idx"].cpu().numpy())
    np.testing.assert_array_equal(crs["stack"], cmp["stack"].cpu().numpy())


@pytest.mark.slow
def test_crs_workload_slice_full_grid(seis):
    """The 1024-CMP CRS line (fold 48, 1500 samples, aperture +-10 CMPs = 1008 traces)
    with the full 21 x 21 x 41 grid, on a slice of 3 central CMPs; the oracle checks a
    seeded sample of rows."""
    ds = synth.workload_crs_line()
    g = seis.to_device(ds)
    central = ds["central"][[0, 511, 1023]]
    ap = seis.crs_aperture(g, central, ds["apm"])
    nb = oracle.aperture(ds, central, ds["apm"])
    assert int(ap.nbr_off[1] - ap.nbr_off[0]) == 1008
    A, B, C = _grids(21, 21, 41)
    got = _run(seis, g, ap, A, B, C, cube=False)
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(ap.rows, 24, replace=False))
    ref = oracle.crs_semblance(ds, nb, A, B, C, rows=rows, want_cube=True)
    rep = parity.check_picks(got["best_idx"][rows], got["best_S"][rows], got["stack"][rows],
                             ref, "crs-line")
    assert rep["pick_agree"] >= 0.9


@pytest.mark.parametrize("shape", ["data1/data2", "data7/data8"])
def test_crs_paper_table1_shapes(seis, shape):
    """A central CMP of the paper's smallest and largest Table 1 shapes, aperture +-1 CMP
    (180 or 3000 traces)."""
    fold, ns = synth.PAPER_SHAPES[shape]
    ds = synth.crs_line(3, fold, ns, 0.004, 0.0, 2400.0, 2, 1, 2.0, seed=310 + fold)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, [1], 12.5)
    nb = oracle.aperture(ds, [1], 12.5)
    A, B, C = _grids(3, 3, 5)
    got = _run(seis, g, ap, A, B, C)
    ref = oracle.crs_semblance(ds, nb, A, B, C, want_cube=True)
    parity.check_cube(got["S"], ref, f"crs {shape}")
    parity.check_picks(got["best_idx"], got["best_S"], got["stack"], ref, f"crs {shape}")


def test_crs_pragmatic_matches_oracle(seis):
    """Central-CMP C search + zero-offset (A, B) search + evaluation over the full aperture,
    against the oracle's composition of the same three steps."""
    ds = synth.crs_line(15, 12, 400, 0.004, 0.0, 1500.0, 3, 1, 2.0, seed=71)
    central, apm = [5, 7, 9], 37.5
    A, B, C = _grids(7, 5, 11)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, central, apm)
    ap_c = seis.crs_aperture(g, central, 0.0)
    ap_z = seis.crs_aperture(g, central, apm, hmax=0.0)
    assert int(ap_z.nbr_off[1] - ap_z.nbr_off[0]) == 7          # one zero-offset trace per CMP
    t = lambda a: torch.from_numpy(a).cuda()
    got = seis.crs_pragmatic(g, ap, ap_c, ap_z, t(A), t(B), t(C), c_zo=float(C[0]))
    torch.cuda.synchronize()
    seis.device_status()
    ref = oracle.crs_pragmatic(ds, central, apm, 0.0, A, B, C, c_zo=C[0])
    ok = ((ref.gap_cmp >= parity.GAP_TOL) & (ref.gap_zo >= parity.GAP_TOL) & ~ref.edge_cmp
          & ~ref.edge_zo)
    th = got["theta"].cpu().numpy()
    assert ok.mean() > 0.8
    np.testing.assert_array_equal(th[ok], ref.theta[ok].astype(np.float32))
    ok &= ~ref.knot
    dS = np.abs(got["S"].cpu().numpy() - ref.S)[ok].max()
    st = got["stack"].cpu().numpy()
    rel = np.linalg.norm((st - ref.stack)[ok]) / np.linalg.norm(ref.stack[ok])
    print(f"[parity] pragmatic CRS: rows compared {ok.mean():.3f}, max dS {dS:.2e}, "
          f"stack rel L2 {rel:.2e}")
    assert dS <= parity.S_TOL and rel <= parity.STACK_TOL


@pytest.mark.parametrize("w", [3, 11])
def test_crs_t0win_matches_oracle(seis, w):
    """CRS with the window over neighbouring output times (64-row blocks, halo lanes)."""
    ds = synth.crs_line(9, 10, 230, 0.004, 0.0, 1500.0, 2, 1, 2.0, seed=81 + w)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, [2, 4, 6], 25.0)
    nb = oracle.aperture(ds, [2, 4, 6], 25.0)
    A, B, C = _grids(5, 3, 7)
    t = lambda a: torch.from_numpy(a).cuda()
    out = seis.crs_semblance_t0win(g, ap, t(A), t(B), t(C), w=w, want_cube=True)
    torch.cuda.synchronize()
    seis.device_status()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.crs_semblance(ds, nb, A, B, C, w=w, want_cube=True, t0_window=True)
    parity.check_cube(got["S"], ref, f"crs t0win w{w}")
    parity.check_picks(got["best_idx"], got["best_S"], got["stack"], ref, f"crs t0win w{w}")
    ia, rem = np.divmod(got["best_idx"], 3 * 7)
    ib, ic = np.divmod(rem, 7)
    np.testing.assert_array_equal(got["best_ABC"], np.stack([A[ia], B[ib], C[ic]], 1))


# --- problems too small to fill the GPU: candidate passes split over CTAs ----------------

def test_split_search_is_bitwise_identical(seis):
    """Two central CMPs (fewer tiles than one wave of the GPU): crs_semblance_ws spreads each
    tile's candidates over several CTAs and merges their argmaxes; every output, the cube
    included, equals crs_semblance's bit for bit, and matches the oracle."""
    ds = synth.crs_line(9, 12, 330, 0.004, 0.0, 1500.0, 2, 1, 2.0, seed=141)
    g = seis.to_device(ds)
    ap = seis.crs_aperture(g, [3, 5], 30.0)
    A, B, C = _grids(7, 5, 13)
    lib = seis.load_library()
    assert lib.seis_search_workspace_size(ap.n_central, ap.max_rows, ap.rows, 7 * 5 * 13) > 0
    t = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    one = seis.crs_semblance(g, ap, t(A), t(B), t(C), w=11, want_cube=True)
    split = seis.crs_semblance(g, ap, t(A), t(B), t(C), w=11, want_cube=True, split=True)
    torch.cuda.synchronize()
    seis.device_status()
    for k in one:
        assert torch.equal(one[k], split[k]), k
    ref = oracle.crs_semblance(ds, oracle.aperture(ds, [3, 5], 30.0), A, B, C, want_cube=True)
    got = {k: v.cpu().numpy() for k, v in split.items()}
    parity.check_cube(got["S"], ref, "crs split")
    parity.check_picks(got["best_idx"], got["best_S"], got["stack"], ref, "crs split")


def test_split_cmp_and_large_problems(seis):
    """CMP: one gather of 300 rows (ten tiles) split, bit-identical to cmp_semblance; a
    workload with a full wave of tiles needs no workspace and takes the plain path; a
    workspace that is too small is refused."""
    lib = seis.load_library()
    ds = synth.cmp_line(1, 20, 300, 0.004, 0.0, 1500.0, 3, 2.0, seed=142)
    g = seis.to_device(ds)
    C = torch.from_numpy(_grids(1, 1, 201)[2]).cuda()
    one = seis.cmp_semblance(g, C, w=11, want_cube=True)
    split = seis.cmp_semblance(g, C, w=11, want_cube=True, split=True)
    torch.cuda.synchronize()
    seis.device_status()
    for k in one:
        assert torch.equal(one[k], split[k]), k
    assert lib.seis_search_workspace_size(4096, 2000, 4096 * 2000, 201) == 0
    need = lib.seis_search_workspace_size(g.ngathers, g.max_rows, g.rows, 201)
    assert need > 0
    ws = torch.empty(need - 16, dtype=torch.uint8, device="cuda")
    out = seis._rows_out(g.traces.device, g.rows, abc=False)
    P = seis._ptr
    rc = lib.cmp_semblance_ws(ctypes.byref(g.descriptor()), P(C), 201, 11, None,
                              P(out["best_idx"]), P(out["best_C"]), P(out["best_S"]),
                              P(out["stack"]), P(ws), ws.numel(), g.rows,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == seis.SEIS_EINVAL and "workspace" in lib.seis_last_error().decode()
