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
