"""Pins of the oracle's Adam step (Sec. 5, "Optimizer") and training-record shuffle (Sec. 3.5).

Adam is pinned by closed forms of the Kingma & Ba recurrences (constant and
alternating gradients); the shuffle by brute-force bijectivity and by the
disjointness of a frame's batches (Sec. 3.3's footnote).
"""
import numpy as np
import pytest

from paper_2106_12372_gb300 import synth


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def test_adam_constant_gradient_closed_form(O):
    # With g constant, m_hat = g and v_hat = g^2 at every t, so each step moves by
    # exactly lr * g / (|g| + eps).
    rng = np.random.default_rng(1)
    g = rng.normal(size=100) * 10.0 ** rng.uniform(-6, 2, 100)
    W0 = rng.normal(size=100)
    W, m, v = W0.copy(), np.zeros(100), np.zeros(100)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        W, m, v = O.adam(W, m, v, g, t, lr=lr, b1=0.9, b2=0.99, eps=eps)
        assert np.allclose(W, W0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-13)


def test_adam_alternating_gradient_step_two(O):
    # g_1 = g, g_2 = -g: m_hat_2 = -(1 - b1) g / (1 + b1), v_hat_2 = g^2.
    b1, b2, lr = 0.9, 0.99, 1e-2
    g = np.array([0.5, -2.0, 3e-3])
    W0 = np.zeros(3)
    W, m, v = O.adam(W0, np.zeros(3), np.zeros(3), g, 1, lr=lr, b1=b1, b2=b2, eps=0.0)
    assert np.allclose(W, -lr * np.sign(g), atol=1e-15)
    W2, _, _ = O.adam(W, m, v, -g, 2, lr=lr, b1=b1, b2=b2, eps=0.0)
    assert np.allclose(W2 - W, lr * (1 - b1) / (1 + b1) * np.sign(g), atol=1e-15)


def test_adam_zero_gradient_keeps_weights(O):
    W0 = np.arange(5.0)
    W, m, v = O.adam(W0, np.zeros(5), np.zeros(5), np.zeros(5), 1)
    assert np.array_equal(W, W0) and np.all(m == 0) and np.all(v == 0)


def test_permutation_bijective_brute_force(O):
    for n in list(range(1, 4097)) + [65536, 16384 * 4 + 7]:
        for seed in (1, 2106) if n <= 4096 else (1, 2, 3):
            p = O.permutation(n, seed)
            assert np.array_equal(np.sort(p), np.arange(n)), n
            a, c = O.lcg_params(n, seed)
            assert np.gcd(a, n) == 1 and 0 <= c < max(n, 1)


def test_batches_are_disjoint_slices_of_one_shuffle(O):
    pool, tgt = synth.make_training_pool(65536, seed=3)
    fs = synth.frame_seed(2106, 0)
    perm = O.permutation(65536, fs)
    seen = []
    for step in range(4):
        rec, t, idx = O.gather(pool, tgt, 16384, fs, step)
        assert np.array_equal(idx, perm[step * 16384:(step + 1) * 16384])
        assert np.array_equal(rec, pool[idx]) and np.array_equal(t, tgt[idx])
        seen.append(idx)
    allidx = np.concatenate(seen)
    assert np.unique(allidx).size == 65536


def test_train_step_is_the_composition_of_its_parts(O):
    dims = synth.layer_dims()
    W0 = synth.xavier_weights(dims, seed=4)
    pool, tgt = synth.make_training_pool(4096, seed=4)
    fs = synth.frame_seed(4, 0)
    st = O.TrainState(W0, dims)
    loss, grad = st.step(pool, tgt, 1024, fs, 1, want_grad=True)
    rec, t, _ = O.gather(pool, tgt, 1024, fs, 1)
    x = O.encode(rec, O.ENC_CHEAP, 1.0)
    y, acts = O.forward(W0, dims, x, keep_acts=True)
    l2, g = O.loss(y, t)
    dW = O.backward(W0, dims, acts, g)
    W1, _, _ = O.adam(W0, np.zeros_like(dW), np.zeros_like(dW), dW, 1)
    assert loss == l2 and np.array_equal(grad, dW) and np.array_equal(st.W, W1) and st.t == 1
