"""Randomised pins of the FP64 oracle (CPU only): on random small gathers (ragged trace
lengths, odd windows, both sampling intervals) the oracle equals an independent pure-Python
loop nest of Eq. 1 / Algorithm 1, and its outputs obey the invariants of Eq. 1."""
import numpy as np
import pytest

import oracle
from tests.dsutil import dataset
from tests.test_oracle import _brute_cmp

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


def _random_gather(seed, fold, ns, dt):
    rng = np.random.default_rng(seed)
    lens = rng.integers(max(2, ns - 8), ns + 9, size=fold)
    traces = [rng.standard_normal(int(L)).astype(np.float32) for L in lens]
    h = rng.uniform(1.0, 500.0, size=fold).astype(np.float32)
    return traces, h, dataset(traces, h, dt, out_ns=[ns])


@settings(max_examples=100, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), fold=st.integers(1, 5), ns=st.integers(16, 40),
       w=st.sampled_from([1, 3, 5, 7]), nc=st.integers(1, 4),
       dt=st.sampled_from([0.002, 0.004]))
def test_oracle_equals_brute_force_on_random_gathers(seed, fold, ns, w, nc, dt):
    traces, h, ds = _random_gather(seed, fold, ns, dt)
    C = oracle.velocity_grid(1400.0, 4500.0, nc).astype(np.float32)
    r = oracle.cmp_semblance(ds, C, w=w)
    ref = _brute_cmp(traces, h, np.float32(dt), C, w, ns)
    np.testing.assert_allclose(r.S, ref, rtol=1e-12, atol=1e-14)


@settings(max_examples=100, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), fold=st.integers(1, 6), ns=st.integers(16, 60),
       w=st.sampled_from([1, 3, 5, 7, 9, 11]), nc=st.integers(1, 6))
def test_oracle_invariants_on_random_gathers(seed, fold, ns, w, nc):
    """0 <= S <= 1 (Cauchy-Schwarz), N <= fold, S = 0 where no trace takes part, the pick is
    the first maximum of its row, and the stack is 0 where N = 0."""
    _, _, ds = _random_gather(seed, fold, ns, 0.004)
    C = oracle.velocity_grid(1400.0, 4500.0, nc).astype(np.float32)
    r = oracle.cmp_semblance(ds, C, w=w)
    assert np.all(r.S >= 0.0) and np.all(r.S <= 1.0 + 1e-12)
    assert np.all((r.N >= 0) & (r.N <= fold))
    assert np.all(r.S[r.N == 0] == 0.0)
    np.testing.assert_array_equal(r.best_idx, np.argmax(r.S, axis=1))
    np.testing.assert_array_equal(r.best_S, r.S.max(axis=1))
    none = r.N[np.arange(len(r.best_idx)), r.best_idx] == 0
    assert np.all(r.stack[none] == 0.0)
