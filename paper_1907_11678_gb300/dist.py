"""Multi-GPU decomposition of the semblance search (one process per GPU).

CMP: gathers are independent (Section 3.5 takes one CDP per task), so each rank takes a
contiguous range of gathers and no data moves between ranks.

CRS: the aperture of a central CDP reaches apm / (CDP spacing) CDPs to each side (Section
2.2), so a line split into contiguous CDP ranges needs, per rank, a halo of that many CDPs
from each neighbour.  Section 3.5 sends the outer region of each grid to its neighbours with
asynchronous messages while the inner region is computed; `crs_search_sharded` does the same
on GPUs:
  1. the halo's metadata (trace lengths, half-offsets, midpoints, output rows and dt per
     gather: a few KB) is exchanged and the rank's extended line (left halo, owned gathers,
     right halo) is laid out in device memory, so gathers may differ in trace length and
     output rows;
  2. the halo's samples are posted as asynchronous point-to-point messages straight into
     their slices of the extended line (NCCL: device buffers; gloo: pinned host buffers,
     then a copy stream);
  3. the central CDPs whose apertures stay inside the owned gathers are searched while the
     messages are in flight, the outer ones once the halo has landed.
Every rank's results equal the single-process search of its central CDPs bit for bit: the
apertures list the same traces in the same order, and the kernels sum in list order.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced [begin, end) of n units for `rank` of `world`."""
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def crs_partition(n_cdp: int, world: int, rank: int, halo: int):
    """Owned CDP range and the range the rank needs (owned plus `halo` CDPs per side,
    clipped to the line)."""
    b, e = shard_range(n_cdp, world, rank)
    return (b, e), (max(0, b - halo), min(n_cdp, e + halo))


def local_part(ds: dict, g0: int, g1: int) -> dict:
    """Gathers [g0, g1) of a dataset dict (synth.py layout) as a dataset dict of their own
    (offsets rebased to 0): what one rank holds of a line before the exchange."""
    goff = np.asarray(ds["gather_off"], np.int64)
    toff = np.asarray(ds["trace_off"], np.int64)
    ooff = np.asarray(ds["out_off"], np.int64)
    t0, t1 = int(goff[g0]), int(goff[g1])
    s0, s1 = int(toff[t0]), int(toff[t1])
    return dict(traces=np.ascontiguousarray(ds["traces"][s0:s1]),
                trace_off=toff[t0:t1 + 1] - s0, h=np.ascontiguousarray(ds["h"][t0:t1]),
                m=np.ascontiguousarray(ds["m"][t0:t1]), gather_off=goff[g0:g1 + 1] - t0,
                out_off=ooff[g0:g1 + 1] - ooff[g0],
                dt=np.ascontiguousarray(np.asarray(ds["dt"], np.float32)[g0:g1]))


class _Block:
    """Host arrays of a contiguous run of gathers: samples, per-trace lengths, h, m, and per
    gather the trace count, output rows and dt."""

    def __init__(self, traces, tlen, h, m, gntr, grows, dt):
        self.traces, self.tlen, self.h, self.m = traces, tlen, h, m
        self.gntr, self.grows, self.dt = gntr, grows, dt

    @classmethod
    def of(cls, ds: dict, g0: int, g1: int) -> "_Block":
        p = local_part(ds, g0, g1)
        return cls(p["traces"].astype(np.float32), np.diff(p["trace_off"]).astype(np.int64),
                   p["h"].astype(np.float32), p["m"].astype(np.float32),
                   np.diff(p["gather_off"]).astype(np.int64),
                   np.diff(p["out_off"]).astype(np.int64), p["dt"].astype(np.float32))

    def header(self) -> np.ndarray:
        return np.array([len(self.traces), len(self.tlen), len(self.gntr)], np.int64)

    def small(self) -> list[np.ndarray]:
        """The metadata arrays, in message order."""
        return [self.tlen, self.h, self.m, self.gntr, self.grows, self.dt]

    @staticmethod
    def empty_small(hdr) -> list[np.ndarray]:
        _, ntr, ng = (int(v) for v in hdr)
        return [np.empty(ntr, np.int64), np.empty(ntr, np.float32), np.empty(ntr, np.float32),
                np.empty(ng, np.int64), np.empty(ng, np.int64), np.empty(ng, np.float32)]


def _p2p(ops):
    """Run a list of (kind, tensor, peer) point-to-point operations at once; returns the
    requests (empty list when there is nothing to do)."""
    if not ops:
        return []
    p2p = [dist.P2POp(dist.isend if k == "send" else dist.irecv, t, peer) for k, t, peer in ops]
    return dist.batch_isend_irecv(p2p)


class HaloExchange:
    """The halo exchange of one rank (see the module docstring).

    `local` holds the rank's owned gathers (a dataset dict, gathers in global order, as
    `local_part` returns); `device` is where the extended line lives.  Construction exchanges
    the metadata (blocking, small) and lays out the extended line: `ext` is a dataset dict of
    tensors on `device` whose traces of the halo gathers are filled only after `wait()`.
    `start()` posts the samples' messages; `wait(stream)` completes them (and, when the
    transport is host memory, copies the halos to the device on a copy stream that `stream`
    then waits for)."""

    def __init__(self, local: dict, n_cdp: int, halo: int, rank: int, world: int,
                 device="cpu", group=None):
        self.rank, self.world, self.halo = rank, world, halo
        self.device = torch.device(device)
        self.group = group
        (ob, oe), _ = crs_partition(n_cdp, world, rank, halo)
        own_n = oe - ob
        if len(local["gather_off"]) - 1 != own_n:
            raise ValueError(f"rank {rank} holds {len(local['gather_off']) - 1} gathers, "
                             f"its share is {own_n}")
        if world > 1 and own_n < halo:
            raise ValueError(f"rank {rank} owns {own_n} gathers, fewer than the halo {halo}")
        backend = dist.get_backend(group) if (world > 1 and dist.is_initialized()) else "gloo"
        # NCCL moves device memory; gloo moves host memory
        self.wire = self.device if backend == "nccl" else torch.device("cpu")
        self.left = rank > 0 and halo > 0 and world > 1
        self.right = rank < world - 1 and halo > 0 and world > 1
        own = _Block.of(local, 0, own_n)
        out_l = _Block.of(local, 0, halo) if self.left else None           # to the left peer
        out_r = _Block.of(local, own_n - halo, own_n) if self.right else None
        self._out = (out_l, out_r)
        # 1a. headers, 1b. metadata arrays (blocking: a few KB)
        hdr_l = np.zeros(3, np.int64)
        hdr_r = np.zeros(3, np.int64)
        self._wait_all(self._exchange(
            [(out_l.header() if self.left else None, hdr_l if self.left else None, rank - 1),
             (out_r.header() if self.right else None, hdr_r if self.right else None, rank + 1)]))
        in_l = _Block.empty_small(hdr_l) if self.left else None
        in_r = _Block.empty_small(hdr_r) if self.right else None
        pairs = []
        if self.left:
            pairs += [(a, b, rank - 1) for a, b in zip(out_l.small(), in_l)]
        if self.right:
            pairs += [(a, b, rank + 1) for a, b in zip(out_r.small(), in_r)]
        self._wait_all(self._exchange(pairs))
        # the extended line: [left halo | owned | right halo]
        parts = []
        if self.left:
            parts.append(_Block(None, *in_l))
        parts.append(own)
        if self.right:
            parts.append(_Block(None, *in_r))
        ns_l = int(hdr_l[0]) if self.left else 0
        ns_r = int(hdr_r[0]) if self.right else 0
        tlen = np.concatenate([p.tlen for p in parts])
        gntr = np.concatenate([p.gntr for p in parts])
        grows = np.concatenate([p.grows for p in parts])
        self.n_left = len(in_l[3]) if self.left else 0
        self.n_own = own_n
        self.n_right = len(in_r[3]) if self.right else 0
        self.global_first = ob - self.n_left
        dev = self.device
        traces = torch.empty(ns_l + len(own.traces) + ns_r, dtype=torch.float32, device=dev)
        traces[ns_l:ns_l + len(own.traces)].copy_(torch.from_numpy(own.traces))
        cat = lambda arrs, dt: torch.from_numpy(np.ascontiguousarray(np.concatenate(arrs), dt))
        self.ext = dict(
            traces=traces,
            trace_off=cat([[0], np.cumsum(tlen)], np.int64).to(dev),
            h=cat([p.h for p in parts], np.float32).to(dev),
            m=cat([p.m for p in parts], np.float32).to(dev),
            gather_off=cat([[0], np.cumsum(gntr)], np.int64).to(dev),
            out_off=cat([[0], np.cumsum(grows)], np.int64).to(dev),
            dt=cat([p.dt for p in parts], np.float32).to(dev))
        self.host_rows = np.concatenate([[0], np.cumsum(grows)]).astype(np.int64)
        self.max_rows = int(grows.max()) if len(grows) else 0
        self.max_trace_samples = int(tlen.max()) if len(tlen) else 0
        self._slices = ((0, ns_l), (len(traces) - ns_r, len(traces)))
        self._reqs = []
        self._stage = None

    def _exchange(self, pairs):
        """Post send/recv of (send array or None, receive array or None, peer) triples on the
        wire device; returns (requests, [(received tensor, numpy destination)])."""
        ops, back = [], []
        for snd, rcv, peer in pairs:
            if snd is not None:
                ops.append(("send", torch.from_numpy(np.ascontiguousarray(snd)).to(self.wire), peer))
            if rcv is not None:
                t = torch.empty(rcv.shape, dtype=torch.from_numpy(rcv[:0]).dtype, device=self.wire)
                ops.append(("recv", t, peer))
                back.append((t, rcv))
        return _p2p(ops), back

    @staticmethod
    def _wait_all(posted):
        reqs, back = posted
        for r in reqs:
            r.wait()
        for t, dst in back:
            dst[...] = t.cpu().numpy()

    def start(self) -> "HaloExchange":
        """Post the halo samples: our boundary gathers out, the neighbours' into the
        extended line (directly, or into pinned host buffers when the wire is host memory)."""
        ops = []
        (l0, l1), (r0, r1) = self._slices
        direct = self.wire == self.device
        self._stage = []
        own0, own1 = l1, r0                                # the owned samples in ext
        sends = {"left": (own0, own0 + (len(self._out[0].traces) if self.left else 0)),
                 "right": (own1 - (len(self._out[1].traces) if self.right else 0), own1)}
        for side, peer, (a, b), blk in (("left", self.rank - 1, (l0, l1), self._out[0]),
                                        ("right", self.rank + 1, (r0, r1), self._out[1])):
            if not getattr(self, side):
                continue
            if direct:                                     # our boundary gathers, in place
                sa, sb = sends[side]
                ops.append(("send", self.ext["traces"][sa:sb], peer))
            else:
                ops.append(("send", torch.from_numpy(blk.traces), peer))
            if direct:
                ops.append(("recv", self.ext["traces"][a:b], peer))
            else:
                buf = torch.empty(b - a, dtype=torch.float32,
                                  pin_memory=self.device.type == "cuda")
                ops.append(("recv", buf, peer))
                self._stage.append((buf, a, b))
        self._reqs = _p2p(ops)
        return self

    def wait(self, stream=None):
        """Complete the halo messages.  Returns a CUDA event that work on the device must
        wait for before reading the halo (None on the CPU)."""
        if self.device.type != "cuda":
            for r in self._reqs:
                r.wait()
            self._reqs = []
            for buf, a, b in self._stage:
                self.ext["traces"][a:b].copy_(buf)
            return None
        copy = torch.cuda.Stream(device=self.device)
        if stream is not None:
            copy.wait_stream(stream)
        with torch.cuda.stream(copy):
            # gloo: blocks until the host buffers are full; NCCL: the copy stream waits
            # for the device-side receives
            for r in self._reqs:
                r.wait()
            self._reqs = []
            for buf, a, b in self._stage:
                self.ext["traces"][a:b].copy_(buf, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(copy)
        self._copy_stream = copy          # keeps the stream (and its pinned sources) alive
        return ev

    def dataset(self) -> dict:
        """The extended line as a dataset dict of numpy arrays (host copy)."""
        return {k: v.cpu().numpy() for k, v in self.ext.items()}


def exchange_halos(local: dict, n_cdp: int, halo: int, rank: int, world: int,
                   device="cpu") -> dict:
    """Blocking halo exchange: the rank's extended line (owned gathers plus up to `halo`
    gathers per side) as a dataset dict of numpy arrays, gathers in global order."""
    ex = HaloExchange(local, n_cdp, halo, rank, world, device=device)
    ex.start()
    ev = ex.wait()
    if ev is not None:
        ev.synchronize()
    return ex.dataset()


def crs_search_sharded(local: dict, n_cdp: int, halo: int, apm: float, A, B, C, w: int = 11,
                       rank: int = 0, world: int = 1, device="cuda", stream=None) -> dict:
    """CRS semblance search of this rank's owned central CDPs on a line split over ranks
    (Section 3.5's inner/outer scheme, see the module docstring).  `local` is the rank's
    owned gathers (local_part); apm must not reach further than `halo` gathers.  Returns the
    search's device outputs (best_idx, best_ABC, best_S, stack) for the owned centrals' rows
    in global order, and 'inner' / 'outer' (the owned central indices searched before and
    after the halo landed)."""
    from . import seis
    dev = torch.device(device)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    ex = HaloExchange(local, n_cdp, halo, rank, world, device=dev)
    g = seis.Gathers(traces=ex.ext["traces"], trace_off=ex.ext["trace_off"], h=ex.ext["h"],
                     m=ex.ext["m"], gather_off=ex.ext["gather_off"], out_off=ex.ext["out_off"],
                     dt=ex.ext["dt"], ngathers=len(ex.host_rows) - 1,
                     ntraces=int(ex.ext["h"].numel()), max_rows=ex.max_rows,
                     max_trace_samples=ex.max_trace_samples, rows=int(ex.host_rows[-1]))
    L, n = ex.n_left, ex.n_own
    # owned centrals whose apertures stay inside the owned gathers
    i0 = halo if ex.left else 0
    i1 = n - halo if ex.right else n
    if i0 >= i1:
        i0 = i1 = n                                   # no inner centrals: all are outer
    blocks = {"inner": [(i0, i1)] if i1 > i0 else [],
              "outer": [(a, b) for a, b in ((0, i0), (i1, n)) if b > a]}
    if i0 == i1 == n:
        blocks["outer"] = [(0, n)]
    rows_of = ex.host_rows[L:L + n + 1] - ex.host_rows[L]
    own_rows = int(rows_of[-1])
    out = dict(best_idx=torch.empty(own_rows, dtype=torch.int32, device=dev),
               best_ABC=torch.empty((own_rows, 3), dtype=torch.float32, device=dev),
               best_S=torch.empty(own_rows, dtype=torch.float32, device=dev),
               stack=torch.empty(own_rows, dtype=torch.float32, device=dev))
    # every aperture reads only midpoints, which the metadata phase delivered
    aps = {k: [(a, b, seis.crs_aperture(g, np.arange(L + a, L + b, dtype=np.int32), apm,
                                        stream=s)) for a, b in v] for k, v in blocks.items()}

    def search(a, b, ap):
        r0, r1 = int(rows_of[a]), int(rows_of[b])
        seis.crs_semblance(g, ap, A, B, C, w=w, stream=s,
                           out={k: v[r0:r1] for k, v in out.items()})
    ex.start()                                        # halo samples in flight ...
    for a, b, ap in aps["inner"]:
        search(a, b, ap)                              # ... while the inner centrals run
    ev = ex.wait(stream=s)
    if ev is not None:
        s.wait_event(ev)
    for a, b, ap in aps["outer"]:
        search(a, b, ap)
    out["inner"] = [(a, b) for a, b, _ in aps["inner"]]
    out["outer"] = [(a, b) for a, b, _ in aps["outer"]]
    out["ext"] = ex
    return out


def max_over_ranks(x: float, device="cpu") -> float:
    """Largest value of x over all ranks (the step time a multi-GPU run reports)."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
