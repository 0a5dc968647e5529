"""Pins of the oracle's weight average (Sec. 3.3, Eq. 2 as read) and reflectance
factorisation (Sec. 5) against definitions independent of its code.

EMA: Eq. 2 as printed does not average (a constant sequence does not map to
itself); the oracle follows the bias-corrected reading
EMA_t = ((1 - a) W_t + a eta_{t-1} EMA_{t-1}) / eta_t, eta_t = 1 - a^t, whose
closed form is the normalised weighted sum  sum_i (1 - a) a^(t-i) W_i / (1 - a^t).

Factorisation: the prediction is the network output times (diffuse + specular
albedo); its weight gradient is checked against central finite differences of
the loss written out here from the forward pass (denominator held fixed, as
the relative L2 loss prescribes), and albedos that sum to one reduce it to the
unfactorised network.
"""
import numpy as np
import pytest

from paper_2106_12372_gb300 import synth


@pytest.fixture(scope="module")
def O():
    from oracle import oracle

    oracle.lib()
    return oracle


def _run_ema(O, seq, alpha, e0=None):
    e = np.zeros_like(seq[0]) if e0 is None else e0.copy()
    out = []
    for t, W in enumerate(seq, start=1):
        e = O.ema(e, W, t, alpha)
        out.append(e)
    return out


@pytest.mark.parametrize("alpha", [0.99, 0.9, 0.5])
def test_ema_of_a_constant_sequence_is_that_constant(O, alpha):
    C = np.random.default_rng(0).normal(size=257)
    for e in _run_ema(O, [C] * 60, alpha):
        assert np.allclose(e, C, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("alpha", [0.99, 0.7])
def test_ema_equals_the_normalised_weighted_sum(O, alpha):
    rng = np.random.default_rng(1)
    seq = [rng.normal(size=100) for _ in range(40)]
    got = _run_ema(O, seq, alpha)
    for T in (1, 2, 5, 40):
        wts = np.array([(1 - alpha) * alpha ** (T - i) for i in range(1, T + 1)])
        ref = np.einsum("i,ij->j", wts, np.array(seq[:T])) / (1 - alpha ** T)
        assert np.allclose(got[T - 1], ref, rtol=1e-11, atol=1e-13), T


def test_ema_first_step_ignores_the_initial_average_and_alpha_zero_tracks_the_weights(O):
    rng = np.random.default_rng(2)
    W1 = rng.normal(size=50)
    assert np.allclose(O.ema(rng.normal(size=50), W1, 1, 0.99), W1, rtol=1e-15, atol=0)
    seq = [rng.normal(size=50) for _ in range(5)]
    for e, W in zip(_run_ema(O, seq, 0.0), seq):
        assert np.allclose(e, W, rtol=0, atol=1e-15)


def test_printed_form_of_eq2_is_not_an_average():
    # the literal formula of the paper, for a constant sequence, drifts away
    # from the constant -- the reason for the bias-corrected reading
    a, C, e = 0.99, 1.0, 0.0
    for t in (1, 2):
        e = (1 - a) / (1 - a ** t) * C + a * (1 - a ** (t - 1)) * e
    assert abs(e - 0.5124) < 1e-3


def test_train_state_tracks_the_average_of_its_weights(O):
    dims = synth.layer_dims()
    W0 = synth.xavier_weights(dims, seed=3)
    pool, tgt = synth.make_training_pool(2048, seed=4)
    st = O.TrainState(W0, dims, ema_alpha=0.99)
    hist = []
    for k in range(4):
        st.step(pool, tgt, 512, synth.frame_seed(9, 0), k)
        hist.append(st.W.copy())
    ref = _run_ema(O, hist, 0.99)[-1]
    assert np.allclose(st.ema, ref, rtol=1e-13, atol=1e-15)


def test_factor_is_the_albedo_sum(O):
    rng = np.random.default_rng(5)
    rec = synth.make_records(64, seed=6)
    y = rng.normal(size=(64, 3))
    f = O.factor(rec, y)
    assert np.allclose(f, y * (rec[:, 8:11].astype(np.float64) + rec[:, 11:14]), rtol=1e-15)


def test_albedos_summing_to_one_reduce_to_the_plain_network(O):
    dims = synth.layer_dims()
    W = synth.xavier_weights(dims, seed=7)
    rec = synth.make_records(300, seed=8)
    rec[:, 11:14] = (1.0 - rec[:, 8:11].astype(np.float64)).astype(np.float32)
    exact = np.abs(rec[:, 8:11].astype(np.float64) + rec[:, 11:14] - 1.0) == 0.0
    y0, y1 = O.infer(W, dims, rec), O.infer(W, dims, rec, refl_factor=True)
    assert np.array_equal(y0[exact], y1[exact])
    assert np.allclose(y0, y1, rtol=1e-7)


def test_factorised_gradient_matches_finite_differences(O):
    dims = synth.layer_dims()
    W0 = synth.xavier_weights(dims, seed=11).astype(np.float64)
    pool, tgt = synth.make_training_pool(256, seed=12)
    fs, batch = synth.frame_seed(13, 0), 64
    st = O.TrainState(W0, dims)
    _, grad = st.step(pool, tgt, batch, fs, 0, refl_factor=True, want_grad=True)
    rec, t, _ = O.gather(pool, tgt, batch, fs, 0)
    x = O.encode(rec)
    f = rec[:, 8:11].astype(np.float64) + rec[:, 11:14]
    yh0 = O.forward(W0, dims, x) * f
    lum = 0.2126 * yh0[:, 0] + 0.7152 * yh0[:, 1] + 0.0722 * yh0[:, 2]
    den = (lum * lum + 0.01)[:, None]

    def surrogate(W):
        yh = O.forward(W, dims, x) * f
        return np.sum((yh - t) ** 2 / den) / (3 * batch)

    rng = np.random.default_rng(14)
    for p in rng.choice(W0.size, 60, replace=False):
        h = 1e-6
        Wp, Wm = W0.copy(), W0.copy()
        Wp[p] += h
        Wm[p] -= h
        fd = (surrogate(Wp) - surrogate(Wm)) / (2 * h)
        assert abs(fd - grad[p]) <= 1e-6 * max(1e-3, abs(grad[p])) + 1e-9, (p, fd, grad[p])
    # the factor matters: without it the gradient differs
    st2 = O.TrainState(W0, dims)
    _, g_plain = st2.step(pool, tgt, batch, fs, 0, want_grad=True)
    assert np.linalg.norm(g_plain - grad) > 1e-3 * np.linalg.norm(grad)
