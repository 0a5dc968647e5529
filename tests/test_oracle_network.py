"""Pins of the oracle's network, loss and backward pass.

* forward: hand-computed integer networks (tests/golden/tiny_nets.json) and the
  all-positive special case, where the ReLU MLP reduces to a product of
  matrices (Sec. 5, "Architecture");
* loss: hand-computed values (tests/golden/loss_cases.json) of Eq. 5 and the
  identity loss = sum g (yhat - y) / 2 that ties the gradient to the value;
* backward: hand-computed gradients and central finite differences in FP64 of
  the linearised objective sum g . y(W) on every weight of a small net and on
  sampled weights of the full-size 64-wide net (Sec. 4).
"""
import json
import os

import numpy as np
import pytest

from paper_2106_12372_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def _flat(Ws):
    return np.concatenate([np.asarray(w, dtype=np.float64).ravel() for w in Ws])


def test_tiny_nets_forward_and_backward(O):
    spec = json.load(open(os.path.join(GOLDEN, "tiny_nets.json")))
    for net in spec["nets"]:
        dims, W = net["dims"], _flat(net["W"])
        for case in net["cases"]:
            x = np.asarray([case["x"]], dtype=np.float64)
            y, acts = O.forward(W, dims, x, keep_acts=True)
            assert np.array_equal(y[0], np.asarray(case["y"], dtype=np.float64)), net["name"]
            if "g" in case:
                dW = O.backward(W, dims, acts, np.asarray([case["g"]], dtype=np.float64))
                assert np.array_equal(dW, _flat(case["dW"])), net["name"]


def test_all_positive_network_is_a_matrix_product(O):
    rng = np.random.default_rng(3)
    dims = synth.layer_dims()
    Ws = [rng.uniform(0.0, 0.1, (dims[l + 1], dims[l])) for l in range(len(dims) - 1)]
    x = rng.uniform(0.0, 1.0, (50, 64))
    y = O.forward(_flat(Ws), dims, x)
    chain = x.T
    for w in Ws:
        chain = w @ chain
    assert np.allclose(y, chain.T, rtol=1e-12, atol=0)


def test_loss_golden_values(O):
    spec = json.load(open(os.path.join(GOLDEN, "loss_cases.json")))
    for case in spec["cases"]:
        val, _ = O.loss(np.asarray(case["yhat"], np.float64), np.asarray(case["target"], np.float32),
                        case["mode"], spec["eps"])
        assert abs(val - case["loss"]) < 1e-14 * max(1.0, abs(case["loss"]))


@pytest.mark.parametrize("mode", [0, 1])
def test_loss_gradient_identity(O, mode):
    # L = (1/3N) sum (yh - y)^2 / D and g = 2 (yh - y) / (3N D) give L = sum g (yh - y) / 2.
    rng = np.random.default_rng(4 + mode)
    yh = rng.normal(size=(200, 3))
    t = rng.lognormal(size=(200, 3)).astype(np.float32)
    val, g = O.loss(yh, t, mode, 0.01)
    assert abs(val - 0.5 * np.sum(g * (yh - t.astype(np.float64)))) < 1e-12 * abs(val)
    # g points from the target to the prediction and vanishes at the target
    assert np.all(np.sign(g) == np.sign(yh - t.astype(np.float64)))
    val0, g0 = O.loss(t.astype(np.float64), t, mode, 0.01)
    assert val0 == 0.0 and np.all(g0 == 0.0)


def _fd_check(O, dims, W, x, g, idx, h=1e-6):
    _, acts = O.forward(W, dims, x, keep_acts=True)
    dW = O.backward(W, dims, acts, g)
    for p in idx:
        Wp, Wm = W.copy(), W.copy()
        Wp[p] += h
        Wm[p] -= h
        fd = (np.sum(g * O.forward(Wp, dims, x)) - np.sum(g * O.forward(Wm, dims, x))) / (2 * h)
        assert abs(fd - dW[p]) <= 1e-6 * max(1.0, abs(dW[p])), (p, fd, dW[p])
    return dW


def test_backward_finite_differences_small_net(O):
    rng = np.random.default_rng(7)
    dims = [6, 5, 4, 3]
    W = rng.normal(size=synth.n_params(dims))
    x = rng.normal(size=(9, 6))
    g = rng.normal(size=(9, 3))
    _fd_check(O, dims, W, x, g, range(W.size))


def test_backward_finite_differences_full_net(O):
    dims = synth.layer_dims()
    W = synth.xavier_weights(dims, seed=11).astype(np.float64)
    rec = synth.make_records(64, seed=12)
    x = O.encode(rec, O.ENC_CHEAP, 1.0)
    t = synth.RadianceField(13)(rec)
    y = O.forward(W, dims, x)
    _, g = O.loss(y, t, 0, 0.01)
    rng = np.random.default_rng(8)
    idx = rng.choice(W.size, 300, replace=False)
    idx = np.concatenate([idx, [0, 4095, 4096, W.size - 1, W.size - 192]])
    _fd_check(O, dims, W, x, g, idx)


def test_backward_width128_net(O):
    dims = synth.layer_dims(width=128, hidden_layers=7)
    assert synth.n_params(dims) == 106880
    W = synth.xavier_weights(dims, seed=21).astype(np.float64)
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, (16, 64))
    g = rng.normal(size=(16, 3))
    _fd_check(O, dims, W, x, g, rng.choice(W.size, 100, replace=False))


def test_output_layer_gradient_closed_form(O):
    # For the last layer, dW_L = sum_rows g H_{L-1}^T with H_{L-1} the last hidden activations.
    rng = np.random.default_rng(10)
    dims = [8, 8, 3]
    W = rng.normal(size=synth.n_params(dims))
    x = rng.normal(size=(20, 8))
    g = rng.normal(size=(20, 3))
    _, acts = O.forward(W, dims, x, keep_acts=True)
    dW = O.backward(W, dims, acts, g)
    W0 = W[:64].reshape(8, 8)
    H1 = np.maximum(x @ W0.T, 0.0)
    assert np.allclose(dW[64:].reshape(3, 8), g.T @ H1, rtol=1e-12, atol=1e-12)
