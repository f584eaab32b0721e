"""Multi-GPU decomposition of the semblance search (one process per GPU).

CMP: gathers are independent (Section 3.5 takes one CDP per task), so each rank takes a
contiguous range of gathers and no data moves between ranks.

CRS: the aperture of a central CDP reaches apm/dm CDPs to each side (Section 2.2), so a
line split into contiguous CDP ranges needs, per rank, a halo of that many CDPs from each
neighbour before the search (Section 3.5 sends the outer region to the neighbouring grids
with asynchronous MPI while the inner region is computed).  `exchange_halos` does that
exchange once with torch.distributed point-to-point messages (NCCL between GPUs, gloo on
CPU); afterwards every rank searches its own central CDPs on its extended line exactly as
on one GPU.
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


def _pack(ds: dict, g0: int, g1: int):
    """Traces of gathers [g0, g1) of a uniform dataset dict as flat tensors."""
    t0, t1 = int(ds["gather_off"][g0]), int(ds["gather_off"][g1])
    s0, s1 = int(ds["trace_off"][t0]), int(ds["trace_off"][t1])
    lens = np.diff(ds["trace_off"][t0:t1 + 1])
    per_gather = np.diff(ds["gather_off"][g0:g1 + 1])
    return (torch.from_numpy(np.ascontiguousarray(ds["traces"][s0:s1])),
            torch.from_numpy(lens.astype(np.int64)),
            torch.from_numpy(per_gather.astype(np.int64)),
            torch.from_numpy(np.ascontiguousarray(ds["h"][t0:t1])),
            torch.from_numpy(np.ascontiguousarray(ds["m"][t0:t1])))


def _send_block(block, peer, device):
    sizes = torch.tensor([len(block[0]), len(block[1]), len(block[2])], dtype=torch.int64,
                         device=device)
    dist.send(sizes, peer)
    for t in block:
        if t.numel():
            dist.send(t.to(device), peer)


def _recv_block(peer, device):
    sizes = torch.empty(3, dtype=torch.int64, device=device)
    dist.recv(sizes, peer)
    ns, nt, ng = (int(v) for v in sizes.tolist())
    shapes = [(ns, torch.float32), (nt, torch.int64), (ng, torch.int64), (nt, torch.float32),
              (nt, torch.float32)]
    out = []
    for n, dt in shapes:
        t = torch.empty(n, dtype=dt, device=device)
        if n:
            dist.recv(t, peer)
        out.append(t.cpu())
    return out


def exchange_halos(local: dict, n_cdp: int, halo: int, rank: int, world: int,
                   device="cpu") -> dict:
    """Exchange the halo CDPs with the neighbouring ranks.

    `local` holds this rank's owned gathers (a dataset dict as in synth.py; its gathers
    are the global gathers of crs_partition's owned range, in order).  Returns a dataset
    dict of the needed range (owned plus up to `halo` gathers per side) in global gather
    order.  Every rank must own at least `halo` gathers.  Even ranks send first and odd
    ranks receive first, so the blocking point-to-point messages cannot deadlock."""
    (ob, oe), _ = crs_partition(n_cdp, world, rank, halo)
    own_n = oe - ob
    if world > 1 and own_n < halo:
        raise ValueError(f"rank {rank} owns {own_n} gathers, fewer than the halo {halo}")
    blocks = {}

    def do_send():
        if rank > 0:                        # the left neighbour's right halo: our first gathers
            _send_block(_pack(local, 0, halo), rank - 1, device)
        if rank < world - 1:                # the right neighbour's left halo: our last gathers
            _send_block(_pack(local, own_n - halo, own_n), rank + 1, device)

    def do_recv():
        if rank > 0:
            blocks["left"] = _recv_block(rank - 1, device)
        if rank < world - 1:
            blocks["right"] = _recv_block(rank + 1, device)

    if halo > 0 and world > 1:
        if rank % 2 == 0:
            do_send()
            do_recv()
        else:
            do_recv()
            do_send()
    own = list(_pack(local, 0, own_n))
    parts = ([blocks["left"]] if "left" in blocks else []) + [own] + \
            ([blocks["right"]] if "right" in blocks else [])
    traces = torch.cat([p[0] for p in parts]).numpy()
    lens = torch.cat([p[1] for p in parts]).numpy()
    per_gather = torch.cat([p[2] for p in parts]).numpy()
    trace_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    gather_off = np.concatenate([[0], np.cumsum(per_gather)]).astype(np.int64)
    G = len(per_gather)
    ns = int(local["out_off"][1] - local["out_off"][0])
    return dict(traces=traces, trace_off=trace_off,
                h=torch.cat([p[3] for p in parts]).numpy(),
                m=torch.cat([p[4] for p in parts]).numpy(),
                gather_off=gather_off, out_off=np.arange(G + 1, dtype=np.int64) * ns,
                dt=np.full(G, local["dt"][0], np.float32))


def max_over_ranks(x: float, device="cpu") -> float:
    """Largest value of x over all ranks (the step time a multi-GPU run reports)."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
