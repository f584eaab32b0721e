"""Multi-rank decomposition on CPU (gloo, world size 2 and 3): CMP sharding covers every
gather once; the CRS halo exchange gives every rank exactly the traces its central CDPs'
apertures need, so its results on its own centrals equal the single-process ones."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1907_11678_gb300 import dist as sdist


def test_shard_range_covers_everything():
    for n in (1, 7, 4096, 10001):
        for world in (1, 2, 3, 8):
            ranges = [sdist.shard_range(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and b - a >= d - c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def test_crs_partition_halo():
    assert sdist.crs_partition(100, 4, 0, 10) == ((0, 25), (0, 35))
    assert sdist.crs_partition(100, 4, 1, 10) == ((25, 50), (15, 60))
    assert sdist.crs_partition(100, 4, 3, 10) == ((75, 100), (65, 100))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    from paper_1907_11678_gb300 import synth
    from tests.dsutil import ragged_line
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_cdp, halo = 24, 3
        full = ragged_line(synth.crs_line(n_cdp, 6, 260, 0.004, 0.0, 1200.0, 2, 1, 2.0, seed=17),
                           seed=5)
        (ob, oe), (nb, ne) = sdist.crs_partition(n_cdp, world, rank, halo)
        local = sdist.local_part(full, ob, oe)              # this rank's owned gathers only
        ext = sdist.exchange_halos(local, n_cdp, halo, rank, world)
        # the extended line is exactly the global gathers [nb, ne)
        want = sdist.local_part(full, nb, ne)
        same = all(np.array_equal(ext[k], want[k]) for k in
                   ("traces", "trace_off", "h", "m", "gather_off", "out_off", "dt"))
        apm = halo * 12.5
        A = np.float32([-2e-4, 0.0, 2e-4]); B = np.float32([0.0, 1e-6]); C = np.float32([3e-7, 8e-7, 1.5e-6])
        central_local = np.arange(ob - nb, oe - nb, dtype=np.int32)
        nb_loc = oracle.aperture(ext, central_local, apm)
        mine = oracle.crs_semblance(ext, nb_loc, A, B, C, want_cube=True)
        # single-process reference for the same centrals
        nb_full = oracle.aperture(full, np.arange(ob, oe, dtype=np.int32), apm)
        ref = oracle.crs_semblance(full, nb_full, A, B, C, want_cube=True)
        ok = (same and np.array_equal(np.diff(nb_loc[0]), np.diff(nb_full[0]))
              and np.array_equal(mine.S, ref.S) and np.array_equal(mine.best_idx, ref.best_idx)
              and np.array_equal(mine.stack, ref.stack))
        t = sdist.max_over_ranks(float(rank) + 0.5)
        q.put((rank, ok, t))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_crs_halo_exchange_matches_single_process(world):
    """Ragged line (uneven trace lengths and output rows per gather): every rank's extended
    line equals the global gathers it needs, and the oracle's CRS search of its central
    CDPs on it equals the single-process search."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok, t in res:
        assert ok, f"rank {rank} differs from the single-process result"
        assert t == world - 0.5            # max over ranks of rank + 0.5


def test_exchange_halos_single_rank_and_zero_halo():
    """One rank (or no halo) exchanges nothing: the rank's own gathers come back unchanged."""
    from paper_1907_11678_gb300 import synth
    ds = synth.crs_line(6, 4, 200, 0.004, 0.0, 500.0, 1, 0, None, seed=12)
    for world, halo in ((1, 3), (1, 0)):
        out = sdist.exchange_halos(ds, 6, halo, 0, world)
        for k in ("out_off", "dt"):
            np.testing.assert_array_equal(out[k], ds[k])
        np.testing.assert_array_equal(out["traces"], ds["traces"])
        np.testing.assert_array_equal(out["trace_off"], ds["trace_off"])
        np.testing.assert_array_equal(out["gather_off"], ds["gather_off"])
        np.testing.assert_array_equal(out["h"], ds["h"])
        np.testing.assert_array_equal(out["m"], ds["m"])


def test_exchange_halos_rejects_small_shards():
    """A rank that owns fewer gathers than the halo cannot serve its neighbours' halos."""
    from paper_1907_11678_gb300 import synth
    ds = synth.crs_line(2, 4, 200, 0.004, 0.0, 500.0, 1, 0, None, seed=13)
    with pytest.raises(ValueError):
        sdist.exchange_halos(ds, 4, 3, 0, 2)
    with pytest.raises(ValueError):                       # not this rank's share of the line
        sdist.exchange_halos(ds, 7, 1, 0, 2)
