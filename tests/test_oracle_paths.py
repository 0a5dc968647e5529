"""Pins of the oracle's training-record pipeline (Sec. 3.3-3.5; termination
heuristic Eqs. 3-4) against hand-worked cases and definitions written out here.
"""
import math

import numpy as np
import pytest

from paper_2106_12372_gb300 import synth


@pytest.fixture(scope="module")
def O():
    from oracle import oracle

    oracle.lib()
    return oracle


def _line_path(steps, pdfcos=1.0, K=None):
    """A path along +z from the camera at the origin: x_1 at z = 1, then the given step lengths."""
    K = K or len(steps) + 1
    v = np.zeros((1, K, 24), np.float32)
    z = 1.0
    v[0, 0, 2] = z
    v[0, :, 14] = pdfcos
    v[0, :, 15] = 1.0
    for j, dz in enumerate(steps, start=1):
        z += dz
        v[0, j, 2] = z
    v[0, :, 19:22] = 1.0
    return v


def test_hand_worked_termination(O):
    # a_0 = 1 / (4 pi); c a_0 = 7.96e-4.  Spread terms 0.01, 0.03: a = 1e-4 after x_2, 1.6e-3 after x_3.
    v = _line_path([0.01, 0.03, 0.5])
    n, _, _, _ = O.paths_terminate(v, 1, 1, (0, 0, 0), 0.01, 1, 0, 0, -1, 0.8)
    assert n[0] == 2
    # with c = 0.1 (c a_0 = 7.96e-3) the sum (0.01 + 0.03 + 0.5)^2 = 0.29 passes only at x_4
    n, _, _, _ = O.paths_terminate(v, 1, 1, (0, 0, 0), 0.1, 1, 0, 0, -1, 0.8)
    assert n[0] == 3
    # pdf |cos| = 4 halves every spread term
    v4 = _line_path([0.01, 0.03, 0.5], pdfcos=4.0)
    v4[0, 0, 15] = 1.0
    n, _, _, _ = O.paths_terminate(v4, 1, 1, (0, 0, 0), 0.01, 1, 0, 0, -1, 0.8)
    assert n[0] == 3  # (0.005 + 0.015)^2 = 4e-4 < 7.96e-4 <= (0.005 + 0.015 + 0.25)^2


def test_termination_is_monotone_in_c(O):
    v = synth.make_paths(40, 30, 8, seed=3)
    prev = None
    for c in (0.001, 0.01, 0.1, 1.0):
        n, _, _, _ = O.paths_terminate(v, 40, 30, synth.PATH_CAMERA, c, 8, 0, 0, -1, 0.8)
        if prev is not None:
            assert np.all(n >= prev)
        prev = n


def test_tiles_select_one_training_pixel_each(O):
    W, H, s, ox, oy = 37, 21, 8, 5, 6
    v = synth.make_paths(W, H, 6, seed=4)
    _, _, _, tiles = O.paths_terminate(v, W, H, synth.PATH_CAMERA, 0.01, s, ox, oy, 3, 0.8)
    tx_n, ty_n = -(-W // s), -(-H // s)
    assert len(tiles) == tx_n * ty_n
    for t, (p, n, m, unb) in enumerate(tiles):
        ty, tx = divmod(t, tx_n)
        px, py = tx * s + ox, ty * s + oy
        if px < W and py < H:
            assert p == py * W + px and unb == int(t % 16 == 3) and m >= n
        else:
            assert p == -1


def test_transport_equals_the_explicit_path_sum(O):
    rng = np.random.default_rng(5)
    K = 7
    v = np.zeros((1, K, 24), np.float32)
    v[0, :, 16:19] = rng.uniform(0, 2, size=(K, 3))
    v[0, :, 19:22] = rng.uniform(0.1, 0.9, size=(K, 3))
    v[0, :, 0:14] = rng.uniform(size=(K, 14))
    tail = np.array([[0.7, 0.2, 1.3]])
    n, m = 2, 5
    recs, tg = O.paths_records(v, [(0, n, m, 0)], tail, 0.8)
    assert recs.shape == (m, 16)
    f = v[0, :, 19:22].astype(np.float64)
    le = v[0, :, 16:19].astype(np.float64)
    for j in range(m):
        ref = np.zeros(3)
        for k in range(j + 1, m + 1):
            ref += np.prod(f[j:k], axis=0) * le[k]
        ref += np.prod(f[j:m], axis=0) * tail[0]
        assert np.allclose(tg[j], ref, rtol=1e-12)
        assert np.array_equal(recs[j, :14], v[0, j, :14]) and not recs[j, 14:].any()


def test_roulette_suffix_is_unbiased(O):
    rng = np.random.default_rng(6)
    K, n, q = 9, 2, 0.7
    base = np.zeros((1, K, 24), np.float32)
    base[0, :, 16:19] = rng.uniform(0, 1, size=(K, 3))
    base[0, :, 19:22] = rng.uniform(0.3, 0.9, size=(K, 3))
    # full-length transport to vertex 0 with nothing beyond the last vertex
    f, le = base[0, :, 19:22].astype(np.float64), base[0, :, 16:19].astype(np.float64)
    full = sum(np.prod(f[0:k], axis=0) * le[k] for k in range(1, K))
    est = []
    for i in range(20000):
        v = base.copy()
        v[0, :, 22] = rng.random(K)
        p_tiles = [(0, n, None, 1)]
        # the roulette's end vertex, as paths_terminate picks it
        m = next(j for j in range(n, K) if j == K - 1 or not (v[0, j, 22] < np.float32(q)))
        _, tg = O.paths_records(v, [(0, n, m, 1)], np.zeros((1, 3)), q)
        est.append(tg[0] if len(tg) else np.zeros(3))
    est = np.array(est)
    sem = est.std(axis=0) / math.sqrt(len(est))
    assert np.all(np.abs(est.mean(axis=0) - full) <= 4 * sem + 1e-12), (est.mean(axis=0), full, sem)


def test_composite_closed_form(O):
    v = synth.make_paths(20, 10, 6, seed=7)
    n, E, T, _ = O.paths_terminate(v, 20, 10, synth.PATH_CAMERA, 1e9, 4, 0, 0, -1, 0.8)  # never terminates early
    assert np.all(n == 5)
    f, le = v[:, :, 19:22].astype(np.float64), v[:, :, 16:19].astype(np.float64)
    ref_E = sum(np.prod(f[:, :j], axis=1) * le[:, j] for j in range(6))
    assert np.allclose(E, ref_E, rtol=1e-12)
    assert np.allclose(T, np.prod(f[:, :5], axis=1), rtol=1e-12)
    rgb = np.random.default_rng(8).uniform(size=(200, 3))
    assert np.allclose(O.paths_composite(E, T, rgb), ref_E + np.prod(f[:, :5], axis=1) * rgb)


def test_decision_checker_accepts_the_definitions_decisions(O):
    v = synth.make_paths(40, 30, 8, seed=4)
    n, _, _, tiles = O.paths_terminate(v, 40, 30, synth.PATH_CAMERA, 0.01, 4, 1, 2, 5, 0.8)
    assert O.paths_check_decisions(v, 40, 30, synth.PATH_CAMERA, 0.01, 4, 1, 2, 5, 0.8, n, tiles) == (True, 0)
    # a path end or a suffix end moved past a clear decision is rejected
    p = int(np.argmax(n < 6))
    n2 = n.copy()
    n2[p] += 1
    assert not O.paths_check_decisions(v, 40, 30, synth.PATH_CAMERA, 0.01, 4, 1, 2, 5, 0.8, n2, tiles)[0]
    t2 = np.array(tiles)
    k = int(np.argmax((t2[:, 0] >= 0) & (t2[:, 3] == 0) & (t2[:, 2] < 7)))
    t2[k, 2] += 1
    assert not O.paths_check_decisions(v, 40, 30, synth.PATH_CAMERA, 0.01, 4, 1, 2, 5, 0.8, n, t2)[0]


def test_decision_checker_accepts_either_side_of_the_threshold(O):
    # c chosen so that c a_0 sits 1e-7 (relative) below a(x_1): FP64 ends the path at x_1; FP32 may
    # take that decision the other way and end it at x_2 (the next decision is clear); x_3 is wrong
    v = _line_path([0.01, 0.5, 0.5])
    s1 = float(v[0, 1, 2]) - float(v[0, 0, 2])
    c = s1 * s1 * (4.0 * math.pi) * (1.0 - 1e-7)
    n, _, _, tiles = O.paths_terminate(v, 1, 1, (0, 0, 0), c, 1, 0, 0, -1, 0.8)
    assert n[0] == 1
    assert 1e-7 < O.termination_band(4)
    s, thr = O._termination_terms(v, (0, 0, 0), c)
    for end, ok in ((1, True), (2, True), (3, False)):
        t = [(0, end, O._suffix_end(s[0], thr[0], end, 4), 0)]
        got = O.paths_check_decisions(v, 1, 1, (0, 0, 0), c, 1, 0, 0, -1, 0.8, np.array([end]), t)
        assert got == (ok, 1 if ok and end != 1 else got[1]), (end, got)
