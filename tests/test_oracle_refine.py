"""Pins of the oracle's refinement (reading c16: projected quasi-Newton gradient ascent in
normalised coordinates) against mathematics, not against the oracle itself (CPU only).

The BFGS update of the inverse curvature estimate, H+ = (I - r s y') H (I - r y s') + r s s'
with r = 1/(s.y), is fixed by facts of the method: the secant condition H+ y = s, symmetry,
positive definiteness when s.y > 0, agreement with the direct update of B = H^-1
(B+ = B - B s s' B / s'Bs + y y' / y's), and termination on a quadratic: after steps along
three Q-conjugate directions with y = Q s, H equals Q^-1 whatever H started as.  The
trajectory is pinned by a two-step case worked by hand: with only the C axis active
(dm = 0 for every trace, so dS/dA = dS/dB = 0), the first trial moves step0 along the
sign of dS/dC, and after an accepted first trial the second is the secant step of
one-dimensional BFGS, d = s g1 / (g0 - g1), capped at length 0.25."""
import numpy as np
import pytest

import oracle
from paper_1907_11678_gb300 import synth


def _spd(rng, scale=1.0):
    M = rng.standard_normal((3, 3))
    return scale * (M @ M.T + 0.3 * np.eye(3))


def _pair(rng):
    """A step s and gradient change y with s.y > 0."""
    while True:
        s, y = rng.standard_normal(3), rng.standard_normal(3)
        if s @ y > 0.2 * np.linalg.norm(s) * np.linalg.norm(y):
            return s, y


def test_bfgs_secant_symmetry_positive_definite():
    rng = np.random.default_rng(11)
    for _ in range(50):
        H = _spd(rng, rng.uniform(0.01, 10.0))
        s, y = _pair(rng)
        Hp = oracle.bfgs_inverse_update(H, s, y)
        np.testing.assert_allclose(Hp @ y, s, rtol=1e-12, atol=1e-12 * np.abs(s).max())
        np.testing.assert_allclose(Hp, Hp.T, rtol=0, atol=1e-13 * np.abs(Hp).max())
        assert np.linalg.eigvalsh((Hp + Hp.T) / 2).min() > 0


def test_bfgs_equals_direct_hessian_update():
    """The inverse form the refinement uses is the inverse of the direct BFGS update."""
    rng = np.random.default_rng(12)
    for _ in range(50):
        H = _spd(rng, rng.uniform(0.1, 3.0))
        s, y = _pair(rng)
        B = np.linalg.inv(H)
        Bs = B @ s
        Bp = B - np.outer(Bs, Bs) / (s @ Bs) + np.outer(y, y) / (y @ s)
        np.testing.assert_allclose(oracle.bfgs_inverse_update(H, s, y), np.linalg.inv(Bp),
                                   rtol=1e-9, atol=1e-12)


def test_bfgs_quadratic_termination():
    """Three steps along Q-conjugate directions (Q's eigenvectors) with y = Q s turn any
    positive definite starting estimate into Q^-1 (the hereditary property)."""
    rng = np.random.default_rng(13)
    for _ in range(20):
        Q = _spd(rng)
        _, V = np.linalg.eigh(Q)
        H = _spd(rng, 0.5)
        for k in range(3):
            s = V[:, k] * rng.uniform(0.5, 2.0) * rng.choice([-1.0, 1.0])
            H = oracle.bfgs_inverse_update(H, s, Q @ s)
        np.testing.assert_allclose(H, np.linalg.inv(Q), rtol=1e-9, atol=1e-11)


def test_bfgs_update_catches_plausible_slips():
    """The checks above fail for a transposed operand or a dropped rho s s' term."""
    rng = np.random.default_rng(14)
    H = _spd(rng)
    s, y = _pair(rng)
    r = 1.0 / (s @ y)
    V = np.eye(3) - r * np.outer(y, s)
    transposed = V @ H @ V.T + r * np.outer(s, s)
    dropped = V.T @ H @ V
    good = oracle.bfgs_inverse_update(H, s, y)
    for wrong in (transposed, dropped):
        assert not np.allclose(wrong @ y, s, rtol=1e-6)
    np.testing.assert_allclose(good @ y, s, rtol=1e-12)


def _c_only_line():
    """CMP gathers as their own CRS apertures (dm = 0): only C moves the traveltime."""
    ds = synth.cmp_line(3, 16, 600, 0.004, 0.0, 1800.0, 3, 4.0, seed=37)
    return ds, oracle.cmp_as_crs(ds)


def test_refine_two_steps_hand_worked():
    ds, nb = _c_only_line()
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    lo, hi = np.array([alo, blo, clo]), np.array([ahi, bhi, chi])
    span = hi - lo
    rows = np.arange(40, 1800, 23)
    rng = np.random.default_rng(5)
    z0 = np.stack([rng.uniform(0.2, 0.8, len(rows)), rng.uniform(0.2, 0.8, len(rows)),
                   rng.uniform(0.15, 0.85, len(rows))], 1)
    th0 = lo + z0 * span
    step0 = 0.05
    r = oracle.crs_refine(ds, nb, th0, lo, hi, steps=2, step0=step0, rows=rows)
    e0 = oracle.crs_eval(ds, nb, th0, rows=rows)
    checked = {"accept-secant": 0, "reject": 0}
    for i in range(len(rows)):
        g0 = e0.grad[i] * span
        assert g0[0] == 0.0 and g0[1] == 0.0          # dm = 0: A and B do not act
        if g0[2] == 0.0:
            continue
        # first trial: H0 = (step0/|g0|) I, so d = step0 * g0/|g0| = step0 * sign(gC) e_C
        z1 = z0[i].copy()
        z1[2] = np.clip(z0[i, 2] + step0 * np.sign(g0[2]), 0.0, 1.0)
        th1 = lo + z1 * span
        np.testing.assert_allclose(r.traj[i, 0, :3], th1, rtol=1e-14, atol=0)
        e1 = oracle.crs_eval(ds, nb, th1[None], rows=rows[i:i + 1])
        np.testing.assert_allclose(r.traj[i, 0, 3], e1.S[0], rtol=1e-12, atol=1e-15)
        accept1 = r.traj[i, 0, 4] == 1.0
        if abs(e1.S[0] - e0.S[i]) > 1e-12:          # a decision not at the rounding level
            assert accept1 == (e1.S[0] >= e0.S[i])
        if not accept1:
            # rejected: the step halves, H unchanged: z2 = z0 + step0/2 * sign(gC) e_C
            z2 = z0[i].copy()
            z2[2] = np.clip(z0[i, 2] + 0.5 * step0 * np.sign(g0[2]), 0.0, 1.0)
            np.testing.assert_allclose(r.traj[i, 1, :3], lo + z2 * span, rtol=1e-14, atol=0)
            checked["reject"] += 1
            continue
        g1 = e1.grad[0] * span
        sc, yc = z1[2] - z0[i, 2], g0[2] - g1[2]
        if not (sc * yc > 1e-6 * abs(sc) * abs(yc)) or g1[2] == 0.0:
            continue                                   # no curvature update: not this case
        # one-dimensional BFGS: H_CC = s/y (the secant condition), so d = s g1 / y; the
        # A and B entries keep H0's value but meet a zero gradient
        d = sc * g1[2] / yc
        if abs(d) > 0.25:
            d = 0.25 * np.sign(d)
        z2 = z1.copy()
        z2[2] = np.clip(z1[2] + d, 0.0, 1.0)
        np.testing.assert_allclose(r.traj[i, 1, :3], lo + z2 * span, rtol=1e-12, atol=0)
        e2 = oracle.crs_eval(ds, nb, (lo + z2 * span)[None], rows=rows[i:i + 1])
        np.testing.assert_allclose(r.traj[i, 1, 3], e2.S[0], rtol=1e-12)
        final = lo + (z2 if r.traj[i, 1, 4] == 1.0 else z1) * span
        if abs(e2.S[0] - e1.S[0]) > 1e-12:
            assert (r.traj[i, 1, 4] == 1.0) == (e2.S[0] >= e1.S[0])
        np.testing.assert_allclose(r.theta[i], final, rtol=1e-12, atol=0)
        checked["accept-secant"] += 1
    assert checked["accept-secant"] >= 10 and checked["reject"] >= 1, checked


def test_refine_trajectory_records_every_trial():
    ds, nb = _c_only_line()
    (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
    lo, hi = np.array([alo, blo, clo]), np.array([ahi, bhi, chi])
    rows = np.arange(100, 1700, 97)
    th0 = np.tile((lo + hi) / 2, (len(rows), 1))
    r = oracle.crs_refine(ds, nb, th0, lo, hi, steps=6, rows=rows)
    for i in range(len(rows)):
        made = ~np.isnan(r.traj[i, :, 3])
        acc = r.traj[i, made, 4] == 1.0
        # the final S is the largest accepted trial's (S never decreases), else the start's
        if acc.any():
            assert r.S[i] == r.traj[i, made, 3][acc][-1]
            assert np.all(np.diff(r.traj[i, made, 3][acc]) >= 0)


# --- starts at the coarse cube's local maxima -------------------------------------------

def _brute_local_max(S, nA, nB, nC):
    """Plain loops over every entry and its grid neighbours."""
    out = np.zeros(S.shape, bool)
    for r in range(S.shape[0]):
        for c in range(S.shape[1]):
            ia, rem = divmod(c, nB * nC)
            ib, ic = divmod(rem, nC)
            ok = True
            for da in (-1, 0, 1):
                for db in (-1, 0, 1):
                    for dc in (-1, 0, 1):
                        a, b, cc = ia + da, ib + db, ic + dc
                        if (da, db, dc) == (0, 0, 0) or not (0 <= a < nA and 0 <= b < nB
                                                             and 0 <= cc < nC):
                            continue
                        n = (a * nB + b) * nC + cc
                        if S[r, n] > S[r, c] or (S[r, n] == S[r, c] and n < c):
                            ok = False
            out[r, c] = ok
    return out


def test_local_max_flags_bruteforce():
    rng = np.random.default_rng(21)
    for nA, nB, nC in [(3, 2, 4), (1, 1, 7), (4, 3, 1), (2, 5, 3), (3, 3, 3)]:
        S = rng.integers(0, 4, size=(6, nA * nB * nC)) / 4.0         # many ties
        np.testing.assert_array_equal(oracle.local_max_flags(S, nA, nB, nC),
                                      _brute_local_max(S, nA, nB, nC))


def test_local_max_starts_hand_worked():
    """Grid 1 x 1 x 5, S = 0.1 0.5 0.2 0.7 0.3: local maxima 3 (0.7) and 1 (0.5) come first,
    then the others by S; with S = 0.5 0.5 0.1 the tie goes to the lower index, so only
    entry 0 is a local maximum.  A 2 x 2 x 2 cube has one local maximum at its largest
    entry."""
    A, B, C = [0.0], [0.0], [10.0, 11.0, 12.0, 13.0, 14.0]
    got = oracle.local_max_starts(np.array([[0.1, 0.5, 0.2, 0.7, 0.3]]), A, B, C, 5)
    np.testing.assert_array_equal(got[:, 0, 2], [13.0, 11.0, 14.0, 12.0, 10.0])
    got = oracle.local_max_starts(np.array([[0.5, 0.5, 0.1]]), A, B, C[:3], 3)
    np.testing.assert_array_equal(got[:, 0, 2], [10.0, 11.0, 12.0])
    flags = oracle.local_max_flags(np.array([[0.5, 0.5, 0.1]]), 1, 1, 3)
    np.testing.assert_array_equal(flags, [[True, False, False]])
    cube = np.array([[0.1, 0.2, 0.3, 0.9, 0.4, 0.5, 0.6, 0.7]])      # 2 x 2 x 2
    flags = oracle.local_max_flags(cube, 2, 2, 2)
    np.testing.assert_array_equal(flags[0], np.arange(8) == 3)
    got = oracle.local_max_starts(cube, [1.0, 2.0], [3.0, 4.0], [5.0, 6.0], 2)
    np.testing.assert_array_equal(got[:, 0], [[1.0, 4.0, 6.0], [2.0, 4.0, 6.0]])
