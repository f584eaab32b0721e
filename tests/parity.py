"""Parity checks of the CUDA path against the FP64 oracle, with the tolerances of the
semblance search:
  - semblance: |dS| <= 1e-4 absolute, except (row, candidate) entries the oracle flags as
    a mask edge on an interpolation knot (reading c5), which must stay below 0.01 %;
  - picked candidates identical, except where the oracle's top-two gap is below 1e-4 or
    the oracle's or the GPU's pick is a flagged entry (a flagged entry elsewhere in the row
    cannot move the pick: if neither pick is flagged, both S values are within tolerance);
  - stacked traces: relative L2 error <= 1e-4 over rows whose picks agree.
"""
import numpy as np

S_TOL = 1e-4
GAP_TOL = 1e-4
STACK_TOL = 1e-4
MAX_EXEMPT = 1e-4          # workload-sized cases
MAX_EXEMPT_SMALL = 5e-3    # tiny cases: entries near the ends of short records


def check_cube(S_gpu, ref, label="", max_exempt=MAX_EXEMPT_SMALL):
    S_gpu = np.asarray(S_gpu, np.float64)
    edge = ref.edge != 0
    frac = edge.mean()
    assert frac <= max_exempt, f"{label}: {frac:.2e} of entries exempt"
    err = np.abs(S_gpu - ref.S)
    exempt_differ = int((err[edge] > S_TOL).sum())
    err[edge] = 0.0
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= S_TOL, f"{label}: max |dS| = {err.max():.3e} at {worst}"
    rep = dict(max_dS=float(err.max()), exempt=float(frac), exempt_differ=exempt_differ)
    print(f"[parity] {label}: {rep}")
    return rep


def check_picks(best_idx, best_S, stack, ref, label="", row_edge=None, edge=None):
    """row_edge [rows]: waive whole rows; edge [rows, ncand] (the oracle's flags): waive a
    row only where the oracle's or the GPU's pick is flagged."""
    best_idx = np.asarray(best_idx)
    best_S = np.asarray(best_S, np.float64)
    stack = np.asarray(stack, np.float64)
    gap = ref.best_S - ref.second_S
    ok_rows = gap >= GAP_TOL
    if row_edge is not None:
        ok_rows &= ~row_edge
    if edge is not None:
        e = np.asarray(edge) != 0
        r = np.arange(len(best_idx))
        gpu_pick = np.clip(best_idx, 0, e.shape[1] - 1)
        ok_rows &= ~(e[r, ref.best_idx] | e[r, gpu_pick])
    same = best_idx == ref.best_idx
    bad = ok_rows & ~same
    assert not bad.any(), (f"{label}: {bad.sum()} picks differ, e.g. rows {np.nonzero(bad)[0][:5]}"
                           f" gpu {best_idx[bad][:5]} ref {ref.best_idx[bad][:5]}")
    # best S at the (agreeing) pick
    dS = np.abs(best_S - ref.best_S)[same]
    assert dS.size == 0 or dS.max() <= S_TOL, f"{label}: best_S max err {dS.max():.3e}"
    ref_st = ref.stack[same]
    num = np.linalg.norm(stack[same] - ref_st)
    den = np.linalg.norm(ref_st)
    rel = num / den if den > 0 else num
    assert rel <= STACK_TOL, f"{label}: stack relative L2 {rel:.3e}"
    rep = dict(pick_agree=float(same.mean()), stack_rel_l2=float(rel),
               waived=float((~ok_rows).mean()))
    print(f"[parity] {label}: {rep}")
    return rep
