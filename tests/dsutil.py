"""Small dataset builders shared by the tests (input construction only, no method
arithmetic)."""
import numpy as np


def dataset(traces_list, h, dt, m=None, gather_sizes=None, out_ns=None):
    """Build a dataset dict from a list of 1-D traces (possibly of different lengths).

    gather_sizes: traces per gather (default: one gather with all traces);
    out_ns: output samples per gather (default: the first trace's length)."""
    lens = [len(t) for t in traces_list]
    trace_off = np.zeros(len(lens) + 1, np.int64)
    trace_off[1:] = np.cumsum(lens)
    if gather_sizes is None:
        gather_sizes = [len(traces_list)]
    gather_off = np.zeros(len(gather_sizes) + 1, np.int64)
    gather_off[1:] = np.cumsum(gather_sizes)
    if out_ns is None:
        out_ns = [lens[gather_off[g]] for g in range(len(gather_sizes))]
    out_off = np.zeros(len(out_ns) + 1, np.int64)
    out_off[1:] = np.cumsum(out_ns)
    G = len(gather_sizes)
    dt = np.broadcast_to(np.asarray(dt, np.float32), (G,)).copy()
    if m is None:
        m = np.zeros(len(lens), np.float32)
    return dict(traces=np.concatenate([np.asarray(t, np.float32) for t in traces_list]),
                trace_off=trace_off, h=np.asarray(h, np.float32), m=np.asarray(m, np.float32),
                gather_off=gather_off, out_off=out_off, dt=dt)


def spike_wavelet(ns, centre, width=2.0):
    """A smooth pulse centred exactly on integer sample `centre` (Gaussian in samples)."""
    s = np.arange(ns, dtype=np.float64)
    return np.exp(-0.5 * ((s - centre) / width) ** 2)


def pythagorean_offsets(n0, max_leg, scale=4):
    """Integers a with n0^2 + (scale*a)^2 a perfect square: returns [(a, m)]."""
    out = []
    for a in range(1, max_leg + 1):
        mm = n0 * n0 + (scale * a) ** 2
        r = int(round(np.sqrt(mm)))
        if r * r == mm:
            out.append((a, r))
    return out


def ragged_line(ds, seed, trim=40, row_trim=30):
    """A copy of a uniform line (synth.crs_line) whose traces are cut to random lengths
    (up to `trim` samples shorter) and whose gathers have random output row counts (up to
    `row_trim` rows fewer): gathers of uneven trace length and rows."""
    rng = np.random.default_rng(seed)
    toff = np.asarray(ds["trace_off"], np.int64)
    n = len(toff) - 1
    lens = np.diff(toff)
    keep = lens - rng.integers(0, trim + 1, n)
    traces = np.concatenate([ds["traces"][toff[i]:toff[i] + keep[i]] for i in range(n)])
    ooff = np.asarray(ds["out_off"], np.int64)
    rows = np.diff(ooff) - rng.integers(0, row_trim + 1, len(ooff) - 1)
    return dict(ds, traces=traces.astype(np.float32),
                trace_off=np.concatenate([[0], np.cumsum(keep)]).astype(np.int64),
                out_off=np.concatenate([[0], np.cumsum(rows)]).astype(np.int64))
