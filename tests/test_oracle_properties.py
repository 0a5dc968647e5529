"""Randomised properties of the oracle (hypothesis; CPU only).

* the shuffle is a bijection of the pool for any pool size and frame seed, and
  the s batches of a frame are disjoint slices of it (Sec. 3.5);
* every one-blob bin holds a non-negative mass, the bins of one value sum to at
  most 1, and to exactly 1 where the kernel lies inside [0, 1] (Sec. 3.6);
* the cheap frequency features stay in [-1, 1] and equal the sine at the points
  where 2^(d+1) x is an integer (Sec. 5, Fig. 7);
* the loss is non-negative and zero exactly at the target (Eq. 5).
"""
import math

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@settings(max_examples=40, deadline=None)
@given(n=st.integers(min_value=1, max_value=20000), seed=st.integers(min_value=0, max_value=2 ** 63 - 1))
def test_shuffle_is_a_bijection(O, n, seed):
    p = O.permutation(n, seed)
    assert p.shape == (n,) and np.array_equal(np.sort(p), np.arange(n))


@settings(max_examples=25, deadline=None)
@given(n=st.integers(min_value=4, max_value=4096), seed=st.integers(min_value=0, max_value=2 ** 32))
def test_batches_partition_a_frame(O, n, seed):
    rng = np.random.default_rng(seed % (2 ** 32))
    pool = rng.random((n, 16), dtype=np.float32)
    tgt = rng.random((n, 3), dtype=np.float32)
    batch = n // 4
    seen = []
    for s in range(4):
        rec, _, idx = O.gather(pool, tgt, batch, seed, s)
        assert np.array_equal(rec, pool[idx])
        seen.append(idx)
    allidx = np.concatenate(seen)
    assert len(np.unique(allidx)) == len(allidx)  # disjoint


@settings(max_examples=200, deadline=None)
@given(s=st.floats(min_value=0.0, max_value=1.0), mode=st.sampled_from([0, 1]))
def test_oneblob_masses(O, s, mode):
    b = np.asarray(O.oneblob(s, 4, mode))
    assert np.all(b >= -1e-15) and b.sum() <= 1.0 + 1e-12
    if mode == 0 and 0.25 <= s <= 0.75:  # the quartic's support [s - 1/4, s + 1/4] lies inside [0, 1]
        assert b.sum() == pytest.approx(1.0, abs=1e-12)


@settings(max_examples=200, deadline=None)
@given(x=st.floats(min_value=0.0, max_value=1.0), d=st.integers(min_value=0, max_value=11))
def test_cheap_frequency_range(O, x, d):
    assert -1.0 - 1e-12 <= O.freq_feature(x, d, 0) <= 1.0 + 1e-12


@settings(max_examples=100, deadline=None)
@given(k=st.integers(min_value=0, max_value=4096), d=st.integers(min_value=0, max_value=11))
def test_cheap_frequency_at_dyadic_points(O, k, d):
    x = (k % (2 ** (d + 1) + 1)) / 2.0 ** (d + 1)
    assert O.freq_feature(x, d, 0) == pytest.approx(math.sin(math.pi * 2.0 ** d * x), abs=1e-12)


@settings(max_examples=100, deadline=None)
@given(seed=st.integers(min_value=0, max_value=2 ** 32 - 1), mode=st.sampled_from([0, 1]))
def test_loss_zero_only_at_the_target(O, seed, mode):
    rng = np.random.default_rng(seed)
    y = rng.uniform(0.0, 3.0, size=(64, 3))
    t = rng.uniform(0.0, 3.0, size=(64, 3)).astype(np.float32)  # targets arrive as FP32
    val, g = O.loss(y, t, mode)
    assert val > 0.0
    val0, g0 = O.loss(t.astype(np.float64), t, mode)
    assert val0 == 0.0 and not np.any(g0)
