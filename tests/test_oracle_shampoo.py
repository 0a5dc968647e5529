"""Pins of the oracle's Shampoo optimiser (the paper's second-order variant,
Sec. 5 "Optimizer"; read as Gupta et al. 2018 with the exponential statistics,
root interval and Adam grafting of Anil et al. 2020).

* on 1x1 matrices the grafted step is exactly Adam's (the oracle's Adam);
* the inverse fourth root: X^4 A = I, X symmetric positive definite;
* diagonal statistics give the closed form D_ij = m_ij (l_i r_j)^(-1/4) up to the
  grafting scale, and the step's Frobenius norm is lr * ||Adam step||_F.
"""
import numpy as np
import pytest

from paper_2106_12372_gb300 import synth


@pytest.fixture(scope="module")
def O():
    from oracle import oracle

    oracle.lib()
    return oracle


def test_scalar_matrices_reduce_to_adam(O):
    rng = np.random.default_rng(0)
    dims = [1, 1, 1]  # two 1x1 "layers"
    W = rng.normal(size=2)
    Wa, ma, va = W.copy(), np.zeros(2), np.zeros(2)
    Ws, ms, vs = W.copy(), np.zeros(2), np.zeros(2)
    Ls, Rs, Ps = [np.zeros((1, 1)), np.zeros((1, 1))], [np.zeros((1, 1)), np.zeros((1, 1))], [None, None]
    for t in range(1, 30):
        G = rng.normal(size=2)
        Wa, ma, va = O.adam(Wa, ma, va, G, t)
        O.shampoo_update(Ws, ms, vs, Ls, Rs, Ps, G, t, dims, eps_rel=0.0, interval=1)
        assert np.allclose(Ws, Wa, rtol=1e-12, atol=1e-14), t


def test_inverse_fourth_root(O):
    rng = np.random.default_rng(1)
    B = rng.normal(size=(64, 64))
    A = B @ B.T + 1e-3 * np.eye(64)
    X = O.inverse_root(A)
    assert np.allclose(X, X.T, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(X) > 0)
    assert np.allclose(np.linalg.matrix_power(X, 4) @ A, np.eye(64), atol=1e-8)


def test_diagonal_statistics_closed_form_and_grafted_norm(O):
    rng = np.random.default_rng(2)
    dims = [4, 3]
    G = np.zeros(12)
    Gm = np.zeros((3, 4))
    Gm[np.arange(3), np.arange(3)] = rng.uniform(0.5, 2.0, size=3)  # G G^T and G^T G diagonal
    G[:] = Gm.ravel()
    W = rng.normal(size=12)
    W0 = W.copy()
    m, v = np.zeros(12), np.zeros(12)
    Ls, Rs, Ps = [np.zeros((3, 3))], [np.zeros((4, 4))], [None]
    O.shampoo_update(W, m, v, Ls, Rs, Ps, G, 1, dims, lr=0.1, eps_rel=0.0, interval=1)
    step = (W0 - W).reshape(3, 4)
    # t = 1: m^ = G, L^ = diag(g^2) (out), R^ = diag(g^2, 0) -> the zero column is regularised only by 1e-30
    d = np.diag(Gm)[:3]
    D = np.zeros((3, 4))
    D[np.arange(3), np.arange(3)] = d * (d * d) ** -0.25 * (d * d) ** -0.25  # = sign(g)
    A = Gm / (np.sqrt(Gm * Gm) + 1e-8)
    expect = 0.1 * D * np.linalg.norm(A) / np.linalg.norm(D)
    assert np.allclose(step, expect, rtol=1e-9, atol=1e-12)
    assert np.linalg.norm(step) == pytest.approx(0.1 * np.linalg.norm(A), rel=1e-12)


def test_shampoo_state_trains(O):
    dims = synth.layer_dims()
    W0 = synth.xavier_weights(dims, seed=3)
    pool, tgt = synth.make_training_pool(4 * 1024, seed=4)
    st = O.ShampooState(W0, dims)
    losses = [st.step(pool, tgt, 1024, synth.frame_seed(5, f), s) for f in range(4) for s in range(4)]
    assert st.t == 16 and np.all(np.isfinite(st.W))
    assert np.median(losses[-4:]) < np.median(losses[:4])
