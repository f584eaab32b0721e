"""Parity checks of the CUDA path against the FP64 oracle, with the tolerances of the
semblance search (semblance |dS| <= 1e-4, stacks relative L2 <= 1e-4, picks identical
where the oracle's top-two gap is at least 1e-4).

Where a trace's participation turns on a test that FP32 rounding may decide either way (a
mask edge on an interpolation knot, or a CRS t0 + A dm or t^2 next to zero; reading c5),
the oracle lists the trace's admissible outcomes and returns, per (row, candidate) entry,
the range [S_lo, S_hi] (and [st_lo, st_hi] for the stack, [N_lo, N_hi] for the trace
count) over every combination of them; other entries have S_lo = S = S_hi.  Every entry
and every row is then checked, none is waived:
  - cube:  S_lo - 1e-4 <= S_gpu <= S_hi + 1e-4 for every entry;
  - picks: for every row, with p the GPU's pick,
      S_lo[p] - 1e-4 <= best_S_gpu <= S_hi[p] + 1e-4   (its S is that of its candidate),
      S_hi[p] + 1e-4 >= max_c S_lo[c]                  (it is an admissible argmax),
    and p equals the oracle's pick wherever the oracle's top-two gap is >= 1e-4 and
    neither pick's entry has a flagged trace;
  - stack: the GPU's stack against the nearest admissible stack of its own pick,
    relative L2 over all rows <= 1e-4.
Entries with more flagged traces than the oracle enumerates stay unresolved (NaN range);
their fraction is capped (MAX_EXEMPT).
"""
import numpy as np

S_TOL = 1e-4
GAP_TOL = 1e-4
STACK_TOL = 1e-4
MAX_EXEMPT = 1e-4          # unresolved entries, workload-sized cases
MAX_EXEMPT_SMALL = 5e-3    # unresolved entries, tiny cases


def _bounds(lo, hi):
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    unres = np.isnan(lo) | np.isnan(hi)
    return np.where(unres, -np.inf, lo), np.where(unres, np.inf, hi), unres


def check_cube(S_gpu, ref, label="", max_exempt=MAX_EXEMPT_SMALL):
    """Every entry of the GPU's cube inside the oracle's admissible range (+- 1e-4)."""
    S_gpu = np.asarray(S_gpu, np.float64)
    lo, hi, unres = _bounds(ref.S_lo, ref.S_hi)
    frac = unres.mean()
    assert frac <= max_exempt, f"{label}: {frac:.2e} of entries unresolved"
    err = np.maximum(np.maximum(lo - S_gpu, S_gpu - hi), 0.0)
    err[unres] = 0.0
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= S_TOL, (f"{label}: S outside the admissible range by {err.max():.3e} "
                                f"at {worst} (gpu {S_gpu[worst]:.6f}, range "
                                f"[{lo[worst]:.6f}, {hi[worst]:.6f}])")
    flagged = np.asarray(ref.edge) != 0
    plain = np.abs(S_gpu - np.asarray(ref.S))[~flagged]
    rep = dict(max_dS=float(plain.max()) if plain.size else 0.0,
               flagged=float(flagged.mean()), unresolved=float(frac),
               flagged_gpu_off_nominal=int((np.abs(S_gpu - ref.S)[flagged] > S_TOL).sum()))
    print(f"[parity] {label}: {rep}")
    return rep


def check_picks(best_idx, best_S, stack, ref, label=""):
    """Every row's pick, best S and stack against the oracle's cube of the same rows (the
    oracle called with want_cube=True, on all rows or on the sampled ones)."""
    best_idx = np.asarray(best_idx).astype(np.int64)
    best_S = np.asarray(best_S, np.float64)
    stack = np.asarray(stack, np.float64)
    nrows, ncand = ref.S_lo.shape
    assert best_idx.shape == (nrows,), f"{label}: {best_idx.shape} picks for {nrows} rows"
    assert np.all((best_idx >= 0) & (best_idx < ncand)), f"{label}: pick index out of range"
    r = np.arange(nrows)
    lo, hi, unres = _bounds(ref.S_lo, ref.S_hi)
    assert unres.mean() <= MAX_EXEMPT_SMALL, f"{label}: {unres.mean():.2e} entries unresolved"
    # (1) the reported best S is the semblance of the reported candidate
    lo_p, hi_p = lo[r, best_idx], hi[r, best_idx]
    e1 = np.maximum(np.maximum(lo_p - best_S, best_S - hi_p), 0.0)
    bad = e1 > S_TOL
    assert not bad.any(), (f"{label}: best_S outside its candidate's range on {bad.sum()} rows, "
                           f"e.g. row {np.nonzero(bad)[0][0]}: {e1.max():.3e}")
    # (2) the reported candidate is an admissible argmax of the row
    row_max_lo = np.max(lo, axis=1)
    short = row_max_lo - (hi_p + S_TOL)
    bad = short > 0
    assert not bad.any(), (f"{label}: pick not an argmax on {bad.sum()} rows, e.g. row "
                           f"{np.nonzero(bad)[0][0]} (S at pick {hi_p[bad][0]:.6f}, row max "
                           f"{row_max_lo[bad][0]:.6f})")
    # (3) identical picks where the oracle's pick is clear and no flagged trace is involved
    flagged = np.asarray(ref.edge) != 0
    gap = ref.best_S - ref.second_S
    clear = (gap >= GAP_TOL) & ~flagged[r, ref.best_idx] & ~flagged[r, best_idx]
    same = best_idx == ref.best_idx
    bad = clear & ~same
    assert not bad.any(), (f"{label}: {bad.sum()} clear picks differ, e.g. rows "
                           f"{np.nonzero(bad)[0][:5]} gpu {best_idx[bad][:5]} "
                           f"ref {ref.best_idx[bad][:5]}")
    # (4) the stack: nearest admissible stack of the GPU's own pick
    slo, shi, sunres = _bounds(ref.st_lo[r, best_idx], ref.st_hi[r, best_idx])
    nearest = np.clip(stack, slo, shi)
    nearest[sunres] = stack[sunres]
    ref_st = np.asarray(ref.stack_at)[r, best_idx]
    num = np.linalg.norm(stack - nearest)
    den = np.linalg.norm(ref_st)
    rel = num / den if den > 0 else num
    assert rel <= STACK_TOL, f"{label}: stack relative L2 {rel:.3e}"
    rep = dict(pick_agree=float(same.mean()), clear_rows=float(clear.mean()),
               stack_rel_l2=float(rel), max_best_S_err=float(e1.max()) if nrows else 0.0)
    print(f"[parity] {label}: {rep}")
    return rep


def check_eval(S_gpu, stack_gpu, N_gpu, ref, label=""):
    """Per-row evaluation at given operators (stack(), the adjoint's S) against the
    oracle's crs_eval ranges: N inside [N_lo, N_hi], S and the stack inside their
    admissible ranges (S +- 1e-4; stack relative L2 <= 1e-4 against the nearest admissible
    value), on every row."""
    S_gpu = np.asarray(S_gpu, np.float64)
    lo, hi, unres = _bounds(ref.S_lo, ref.S_hi)
    assert unres.mean() <= MAX_EXEMPT_SMALL, f"{label}: {unres.mean():.2e} rows unresolved"
    e = np.maximum(np.maximum(lo - S_gpu, S_gpu - hi), 0.0)
    assert e.max() <= S_TOL, f"{label}: S outside its range by {e.max():.3e} at row {e.argmax()}"
    if N_gpu is not None:
        N_gpu = np.asarray(N_gpu)
        bad = (N_gpu < ref.N_lo) | (N_gpu > ref.N_hi)
        assert not bad.any(), f"{label}: N outside its range on {bad.sum()} rows"
    rel = None
    if stack_gpu is not None:
        stack_gpu = np.asarray(stack_gpu, np.float64)
        slo, shi, sunres = _bounds(ref.st_lo, ref.st_hi)
        nearest = np.clip(stack_gpu, slo, shi)
        nearest[sunres] = stack_gpu[sunres]
        den = np.linalg.norm(ref.stack)
        rel = np.linalg.norm(stack_gpu - nearest) / den if den > 0 else 0.0
        assert rel <= STACK_TOL, f"{label}: stack relative L2 {rel:.3e}"
    flagged = ref.S_lo != ref.S_hi
    rep = dict(max_dS=float(np.abs(S_gpu - ref.S)[~flagged].max()) if (~flagged).any() else 0.0,
               flagged=float(flagged.mean()), stack_rel_l2=rel)
    print(f"[parity] {label}: {rep}")
    return rep
