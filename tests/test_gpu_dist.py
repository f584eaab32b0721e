"""The sharded CRS search on the CUDA path: two gloo ranks share the one GPU, each holds
only its own gathers of a ragged line, exchanges halos (dist.crs_search_sharded: metadata,
then the samples in flight while the inner central CDPs are searched), and searches its
central CDPs on its extended line.  Each rank's results must equal the single-process CUDA
search of the same central CDPs bit for bit, and match the oracle on sampled rows.  The
ranks' kernels never wait on one another: every exchange is a host-side message."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gpu_worker(rank, world, port, q):
    try:
        import torch
        import torch.distributed as dist
        import oracle
        from paper_1907_11678_gb300 import dist as sdist, seis, synth
        from tests import parity
        from tests.dsutil import ragged_line
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        n_cdp, halo, apm = 40, 3, 37.5
        full = ragged_line(synth.crs_line(n_cdp, 12, 400, 0.004, 0.0, 1500.0, 3, 1, 2.0,
                                          seed=91), seed=92)
        (alo, ahi), (blo, bhi), (clo, chi) = synth.crs_ranges()
        A = seis.linear_grid(alo, ahi, 5)
        B = seis.linear_grid(blo, bhi, 3)
        C = seis.linear_grid(clo, chi, 7)
        (ob, oe), _ = sdist.crs_partition(n_cdp, world, rank, halo)
        # sharded: this rank holds only its own gathers
        got = sdist.crs_search_sharded(sdist.local_part(full, ob, oe), n_cdp, halo, apm, A, B,
                                       C, w=11, rank=rank, world=world, device="cuda")
        torch.cuda.synchronize()
        seis.device_status()
        # the single-process CUDA search of the same central CDPs on the whole line
        g = seis.to_device(full)
        ap = seis.crs_aperture(g, np.arange(ob, oe, dtype=np.int32), apm)
        ref = seis.crs_semblance(g, ap, A, B, C, w=11)
        torch.cuda.synchronize()
        keys = ("best_idx", "best_ABC", "best_S", "stack")
        bitwise = all(torch.equal(got[k], ref[k]) for k in keys)
        # the oracle on sampled rows of this rank's centrals
        rows = np.sort(np.random.default_rng(rank).choice(ap.rows, 48, replace=False))
        An, Bn, Cn = (t.cpu().numpy() for t in (A, B, C))
        ro = oracle.crs_semblance(full, oracle.aperture(full, np.arange(ob, oe), apm), An, Bn,
                                  Cn, rows=rows, want_cube=True)
        h = {k: got[k].cpu().numpy() for k in keys}
        parity.check_picks(h["best_idx"][rows], h["best_S"][rows], h["stack"][rows], ro,
                           f"sharded rank {rank}")
        q.put((rank, bitwise, got["inner"], got["outer"], None))
        dist.destroy_process_group()
    except Exception as e:                     # report, so the parent does not wait forever
        import traceback
        q.put((rank, False, None, None, traceback.format_exc()))


def test_sharded_crs_search_matches_single_process_bitwise():
    import torch.multiprocessing as mp
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1907_11678_gb300 import build
    build.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
    for rank, bitwise, inner, outer, err in sorted(res):
        assert err is None, f"rank {rank}:\n{err}"
        assert bitwise, f"rank {rank}: sharded results differ from the single-process run"
        # both ranks have interior centrals searched while their halo was in flight
        assert inner and outer, (rank, inner, outer)
    for p in procs:
        assert p.exitcode == 0
