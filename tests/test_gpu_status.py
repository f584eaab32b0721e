"""Failure detection without a GPU fault: a bounded device wait that nothing completes
gives up, the status word reports SEIS_ETIMEOUT, and the context stays usable."""
import time

import numpy as np
import pytest

from paper_1907_11678_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_gives_up_and_reports():
    from paper_1907_11678_gb300 import build, seis
    build.build()
    seis.device_status()                              # clear anything earlier
    t0 = time.perf_counter()
    seis.selftest_wait_timeout(10000)                 # 10 ms limit on a wait nobody ends
    with pytest.raises(seis.SeisError) as e:
        seis.device_status()
    elapsed = time.perf_counter() - t0
    assert e.value.code == seis.SEIS_ETIMEOUT
    assert elapsed < 5.0
    seis.device_status()                              # cleared
    # the context is still usable: a normal search runs and checks clean
    ds = synth.cmp_line(2, 8, 200, 0.004, 0.0, 1000.0, 2, 2.0, seed=3)
    g = seis.to_device(ds)
    C = seis.velocity_grid(1400.0, 4500.0, 21)
    out = seis.cmp_semblance(g, C, w=11)
    torch.cuda.synchronize()
    seis.device_status()
    assert np.isfinite(out["best_S"].cpu().numpy()).all()


def test_fast_traveltime_arithmetic_error_bound():
    """The approximate square root and reciprocal of the traveltime stay within 2^-21
    relative error (measured on every float in [1, 4)); with the cancellation-free moveout
    D = C q / (sqrt(n^2 + C q) + n) this moves u = n + D by at most about 3 * 2^-21 * D
    samples, below the 1e-3-sample mask-edge tolerance of the parity checks for any moveout
    under 600 samples, and far below it for the window's interpolation fraction."""
    from paper_1907_11678_gb300 import build, seis
    build.build()
    es, er = seis.selftest_fast_math()
    torch.cuda.synchronize()
    print(f"[fast-math] max relative error: sqrt {es:.3e} ({np.log2(es):.2f} bits), "
          f"rcp {er:.3e} ({np.log2(er):.2f} bits)")
    assert 0 < es <= 2.0 ** -21 and 0 < er <= 2.0 ** -21
