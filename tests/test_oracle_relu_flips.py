"""Pins the FP64 restatement in tests/relu_flips.py to the oracle: its batch
gradient equals the oracle's, and a decision taken the other way changes the
gradient by exactly that record's contribution with that unit gated the
other way (checked against a direct recomputation)."""
import numpy as np
import pytest

from paper_2106_12372_gb300 import synth
import relu_flips as RF


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("pad", [1.0, 0.0])
def test_batch_gradient_equals_the_oracle(O, pad):
    dims = synth.layer_dims()
    w = synth.xavier_weights(dims, seed=71)
    pool, tgt = synth.make_training_pool(2048, seed=72)
    fs = synth.frame_seed(73, 0)
    st = O.TrainState(w, dims)
    _, ref = st.step(pool, tgt, 1024, fs, 0, pad_value=pad, want_grad=True)
    rec, tg, _ = O.gather(pool, tgt, 1024, fs, 0)
    g = RF.batch_grad(w, dims, O.encode(rec, 0, pad), tg)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


def test_a_flip_is_one_records_gated_contribution(O):
    dims = synth.layer_dims()
    w = synth.xavier_weights(dims, seed=74)
    pool, tgt = synth.make_training_pool(512, seed=75)
    rec, tg, _ = O.gather(pool, tgt, 512, synth.frame_seed(76, 0), 0)
    x = np.asarray(O.encode(rec, 0, 1.0), np.float64)
    t = np.asarray(tg, np.float64)
    Ws = RF._mats(w, dims)
    full = RF._grad_rows(Ws, x, t, 512, 0.01)
    rng = np.random.default_rng(77)
    flips = []
    for _ in range(12):  # single-record changes, computed from that record alone
        l, r, u = int(rng.integers(0, 5)), int(rng.integers(0, 512)), int(rng.integers(0, 64))
        dg = (RF._grad_rows(Ws, x[r:r + 1], t[r:r + 1], 512, 0.01, flip=(l, 0, u))
              - RF._grad_rows(Ws, x[r:r + 1], t[r:r + 1], 512, 0.01))
        flips.append((l, r, u, dg))
    l, r, u, dg = flips[5]
    # the same change from the whole batch with that decision inverted
    flipped = RF._grad_rows(Ws, x, t, 512, 0.01, flip=(l, r, u))
    assert np.allclose(flipped - full, dg, rtol=1e-9, atol=1e-15)
    # explain() recovers a planted flip
    adj, used = RF.explain(full + dg, full, flips)
    assert used >= 1 and np.abs(adj - (full + dg)).max() <= 1e-12 * np.abs(full).max()
