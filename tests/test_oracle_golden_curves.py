"""The stored oracle loss curves reproduce: the first steps of the width-128
curves in tests/golden/width128_curve_fp64.json, recomputed by the oracle now
(realization 0 and one perturbed realization)."""
import json
import os

import numpy as np
import pytest

from paper_2106_12372_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "width128_curve_fp64.json")


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("k", [0, 2])
def test_width128_curve_golden_reproduces(O, k):
    gold = json.load(open(GOLD))
    dims = synth.layer_dims(width=128, hidden_layers=7)
    w0 = synth.xavier_weights(dims, seed=56).astype(np.float64)
    if k:
        w0 = w0 * (1.0 + 1e-7 * np.random.default_rng(k).standard_normal(w0.size))
    pool, tgt = synth.make_training_pool(4 * 2048, seed=57)
    st = O.TrainState(w0, dims)
    got = [st.step(pool, tgt, 2048, synth.frame_seed(58, f), s) for f in range(2) for s in range(4)]
    np.testing.assert_allclose(got, gold["realizations"][k][:8], rtol=1e-9)
    assert gold["medians"][k] == pytest.approx(float(np.median(gold["realizations"][k])))
