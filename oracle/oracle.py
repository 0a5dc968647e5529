"""Python access to the FP64 CPU oracle (``nrc_oracle.cpp``).

TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
benchmark's CPU-baseline and reference legs may import this module.  The CUDA
library and its binding never import it; the two implementations share no
code.

Every function takes numpy arrays, promotes FP32 inputs to FP64 exactly as the
C code does, and returns FP64 results.  See the C source for the passage of
the paper each step follows.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrc_oracle.cpp")
# NRC_ORACLE_SANITIZE=1: the oracle built with AddressSanitizer and
# UndefinedBehaviorSanitizer (load it with libasan preloaded)
_SANITIZE = os.environ.get("NRC_ORACLE_SANITIZE", "") == "1"
_SAN_FLAGS = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-g"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_san.so" if _SANITIZE else "liboracle.so")
_lock = threading.Lock()
_lib = None

ENC_CHEAP, ENC_EXACT = 0, 1
LOSS_LUMINANCE, LOSS_PER_CHANNEL = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no -ffast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp] + (_SAN_FLAGS if _SANITIZE else []))
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64, u64, i32, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
            sig = {
                "oracle_abi_version": (i32, []),
                "oracle_lcg_params": (None, [i64, u64, P, P]),
                "oracle_permutation": (None, [i64, u64, P]),
                "oracle_gather": (None, [P, P, i64, i64, u64, i32, P, P, P]),
                "oracle_tri": (f64, [f64]),
                "oracle_quartic": (f64, [f64]),
                "oracle_quartic_cdf": (f64, [f64]),
                "oracle_freq_feature": (f64, [f64, i32, i32]),
                "oracle_oneblob": (None, [f64, i32, i32, P]),
                "oracle_encode": (None, [P, i64, i32, f64, P]),
                "oracle_forward": (None, [P, P, i32, P, i64, P, P]),
                "oracle_loss": (f64, [P, P, i64, i32, f64, P]),
                "oracle_backward": (None, [P, P, i32, P, P, i64, P]),
                "oracle_adam": (None, [P, P, P, P, i64, i64, f64, f64, f64, f64]),
                "oracle_infer": (None, [P, P, i32, P, i64, i32, f64, i32, P]),
                "oracle_train_step": (f64, [P, P, P, P, P, i32, P, P, i64, i64, u64, i32, i32, f64, i32, f64,
                                            f64, f64, f64, f64, i32, P]),
                "oracle_ema": (None, [P, P, i64, i64, f64]),
                "oracle_factor": (None, [P, i64, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(dims, dtype=np.int32)


# ---------------------------------------------------------------- primitives
def tri(x: float) -> float:
    return lib().oracle_tri(float(x))


def quartic(x: float) -> float:
    return lib().oracle_quartic(float(x))


def quartic_cdf(y: float) -> float:
    return lib().oracle_quartic_cdf(float(y))


def freq_feature(x: float, d: int, enc_mode: int = ENC_CHEAP) -> float:
    return lib().oracle_freq_feature(float(x), int(d), int(enc_mode))


def oneblob(s: float, k: int = 4, enc_mode: int = ENC_CHEAP) -> np.ndarray:
    out = np.zeros(k, dtype=np.float64)
    lib().oracle_oneblob(float(s), int(k), int(enc_mode), _p(out))
    return out


# ------------------------------------------------------------------- steps
def lcg_params(n_pool: int, frame_seed: int) -> tuple[int, int]:
    a, c = ctypes.c_uint64(), ctypes.c_uint64()
    lib().oracle_lcg_params(int(n_pool), int(frame_seed), ctypes.byref(a), ctypes.byref(c))
    return a.value, c.value


def permutation(n_pool: int, frame_seed: int) -> np.ndarray:
    out = np.zeros(n_pool, dtype=np.int64)
    lib().oracle_permutation(int(n_pool), int(frame_seed), _p(out))
    return out


def gather(pool, target, batch: int, frame_seed: int, step: int):
    pool, target = _f32(pool), _f32(target)
    rec = np.zeros((batch, 16), dtype=np.float32)
    tgt = np.zeros((batch, 3), dtype=np.float32)
    idx = np.zeros(batch, dtype=np.int64)
    lib().oracle_gather(_p(pool), _p(target), pool.shape[0], int(batch), int(frame_seed), int(step), _p(rec),
                        _p(tgt), _p(idx))
    return rec, tgt, idx


def encode(rec, enc_mode: int = ENC_CHEAP, pad_value: float = 1.0) -> np.ndarray:
    rec = _f32(rec).reshape(-1, 16)
    out = np.zeros((rec.shape[0], 64), dtype=np.float64)
    lib().oracle_encode(_p(rec), rec.shape[0], int(enc_mode), float(pad_value), _p(out))
    return out


def forward(W, dims, x, keep_acts: bool = False):
    W, x, d = _f64(W), _f64(x), _dims(dims)
    n = x.shape[0]
    L = len(dims) - 1
    y = np.zeros((n, dims[-1]), dtype=np.float64)
    acts = np.zeros(sum(n * dims[l] for l in range(L)), dtype=np.float64) if keep_acts else None
    lib().oracle_forward(_p(W), _p(d), L, _p(x), n, _p(y), _p(acts))
    return (y, acts) if keep_acts else y


def loss(yhat, target, loss_mode: int = LOSS_LUMINANCE, eps: float = 0.01):
    yhat, target = _f64(yhat), _f32(target)
    g = np.zeros_like(yhat)
    val = lib().oracle_loss(_p(yhat), _p(target), yhat.shape[0], int(loss_mode), float(eps), _p(g))
    return val, g


def backward(W, dims, acts, g) -> np.ndarray:
    W, acts, g, d = _f64(W), _f64(acts), _f64(g), _dims(dims)
    dW = np.zeros_like(W)
    lib().oracle_backward(_p(W), _p(d), len(dims) - 1, _p(acts), _p(g), g.shape[0], _p(dW))
    return dW


def adam(W, m, v, g, t: int, lr=1e-2, b1=0.9, b2=0.99, eps=1e-8):
    """Returns updated copies (W, m, v) after Adam step t (t >= 1)."""
    W, m, v, g = _f64(W).copy(), _f64(m).copy(), _f64(v).copy(), _f64(g)
    lib().oracle_adam(_p(W), _p(m), _p(v), _p(g), W.size, int(t), lr, b1, b2, eps)
    return W, m, v


def infer(W, dims, rec, enc_mode: int = ENC_CHEAP, pad_value: float = 1.0, refl_factor: bool = False) -> np.ndarray:
    W, d, rec = _f64(W), _dims(dims), _f32(rec).reshape(-1, 16)
    y = np.zeros((rec.shape[0], dims[-1]), dtype=np.float64)
    lib().oracle_infer(_p(W), _p(d), len(dims) - 1, _p(rec), rec.shape[0], int(enc_mode), float(pad_value),
                       int(bool(refl_factor)), _p(y))
    return y


def ema(ema_prev, W, t: int, alpha: float = 0.99) -> np.ndarray:
    """The weight average after step t >= 1 (Eq. 2, bias-corrected reading)."""
    out = _f64(ema_prev).copy()
    lib().oracle_ema(_p(out), _p(_f64(W)), out.size, int(t), float(alpha))
    return out


def factor(rec, y) -> np.ndarray:
    """y (n x 3) times the records' diffuse + specular albedo, per channel."""
    rec, out = _f32(rec).reshape(-1, 16), _f64(y).copy()
    lib().oracle_factor(_p(rec), rec.shape[0], _p(out))
    return out


class TrainState:
    """FP64 master weights, Adam moments and step counter of one cache."""

    def __init__(self, W, dims, ema_alpha: float | None = None):
        self.dims = list(dims)
        self.W = _f64(W).copy()
        self.m = np.zeros_like(self.W)
        self.v = np.zeros_like(self.W)
        self.t = 0
        self.ema_alpha = ema_alpha
        self.ema = self.W.copy() if ema_alpha is not None else None

    def step(self, pool, target, batch: int, frame_seed: int, step: int, enc_mode=ENC_CHEAP, pad_value=1.0,
             loss_mode=LOSS_LUMINANCE, loss_eps=0.01, lr=1e-2, b1=0.9, b2=0.99, adam_eps=1e-8,
             refl_factor: bool = False, want_grad: bool = False):
        pool, target = _f32(pool), _f32(target)
        t = ctypes.c_int64(self.t)
        grad = np.zeros_like(self.W) if want_grad else None
        val = lib().oracle_train_step(_p(self.W), _p(self.m), _p(self.v), ctypes.byref(t), _p(_dims(self.dims)),
                                      len(self.dims) - 1, _p(pool), _p(target), pool.shape[0], int(batch),
                                      int(frame_seed), int(step), int(enc_mode), float(pad_value), int(loss_mode),
                                      float(loss_eps), lr, b1, b2, adam_eps, int(bool(refl_factor)), _p(grad))
        self.t = t.value
        if self.ema is not None:
            lib().oracle_ema(_p(self.ema), _p(self.W), self.W.size, self.t, float(self.ema_alpha))
        return (val, grad) if want_grad else val


# ----------------------------------------------------------------- Shampoo --
# The second-order optimiser the paper evaluated against Adam (Sec. 5,
# "Optimizer": Shampoo, Gupta et al. 2018, with the refinements of Anil et al.
# 2020).  The paper gives no constants; the reading implemented here:
#   per weight matrix W_l (out x in) with gradient G_l,
#     m   <- b1 m + (1 - b1) G                      (momentum, as Adam's)
#     v   <- b2 v + (1 - b2) G*G                    (Adam's second moment, for grafting)
#     L_l <- b2 L_l + (1 - b2) G G^T,  R_l <- b2 R_l + (1 - b2) G^T G
#     every `interval` steps (from step 1):
#       P_L = (L_l / (1 - b2^t) + eps_l I)^(-1/4),  eps_l = eps_rel * tr(.)/n, same for R
#     D   = P_L  m^  P_R,   m^ = m / (1 - b1^t)
#     A   = m^ / (sqrt(v / (1 - b2^t)) + adam_eps)  (Adam's step)
#     W_l <- W_l - lr * D * ||A||_F / ||D||_F        (layer-wise grafting of Adam's step size)
# For 1x1 matrices the step is exactly Adam's.  Inverse roots by a symmetric
# eigendecomposition in FP64 (numpy.linalg.eigh).


def inverse_root(A: np.ndarray, p: int = 4) -> np.ndarray:
    """A^(-1/p) of a symmetric positive definite matrix (FP64 eigendecomposition)."""
    w, V = np.linalg.eigh(np.asarray(A, dtype=np.float64))
    return (V * w ** (-1.0 / p)) @ V.T


def shampoo_update(W, m, v, Ls, Rs, Ps, G, t: int, dims, lr=1e-2, b1=0.9, b2=0.99, adam_eps=1e-8,
                   eps_rel=1e-4, interval: int = 4):
    """One Shampoo step (t >= 1) on flat FP64 arrays W, m, v and per-layer lists
    Ls, Rs (statistics) and Ps (list of [P_L, P_R] or None); updated in place."""
    off = 0
    recompute = (t - 1) % interval == 0
    m *= b1
    m += (1.0 - b1) * G
    v *= b2
    v += (1.0 - b2) * G * G
    for l in range(len(dims) - 1):
        n_out, n_in = dims[l + 1], dims[l]
        sl = slice(off, off + n_out * n_in)
        off += n_out * n_in
        Gl = G[sl].reshape(n_out, n_in)
        Ls[l] *= b2
        Ls[l] += (1.0 - b2) * Gl @ Gl.T
        Rs[l] *= b2
        Rs[l] += (1.0 - b2) * Gl.T @ Gl
        if recompute or Ps[l] is None:
            roots = []
            for S in (Ls[l], Rs[l]):
                Sh = S / (1.0 - b2 ** t)
                n = Sh.shape[0]
                roots.append(inverse_root(Sh + (eps_rel * np.trace(Sh) / n + 1e-30) * np.eye(n)))
            Ps[l] = roots
        mh = m[sl].reshape(n_out, n_in) / (1.0 - b1 ** t)
        D = Ps[l][0] @ mh @ Ps[l][1]
        A = mh / (np.sqrt(v[sl].reshape(n_out, n_in) / (1.0 - b2 ** t)) + adam_eps)
        nd = np.linalg.norm(D)
        W[sl] -= lr * (D * (np.linalg.norm(A) / nd if nd > 0 else 0.0)).ravel()


class ShampooState:
    """FP64 weights and Shampoo state of one cache (training step as TrainState.step)."""

    def __init__(self, W, dims, lr=1e-2, eps_rel=1e-4, interval: int = 4):
        self.dims = list(dims)
        self.W = _f64(W).copy()
        self.m = np.zeros_like(self.W)
        self.v = np.zeros_like(self.W)
        self.Ls = [np.zeros((dims[l + 1], dims[l + 1])) for l in range(len(dims) - 1)]
        self.Rs = [np.zeros((dims[l], dims[l])) for l in range(len(dims) - 1)]
        self.Ps = [None] * (len(dims) - 1)
        self.t = 0
        self.lr, self.eps_rel, self.interval = lr, eps_rel, interval

    def step(self, pool, target, batch: int, frame_seed: int, step: int, enc_mode=ENC_CHEAP, pad_value=1.0,
             loss_mode=LOSS_LUMINANCE, loss_eps=0.01, want_grad: bool = False):
        rec, tgt, _ = gather(pool, target, batch, frame_seed, step)
        x = encode(rec, enc_mode, pad_value)
        y, acts = forward(self.W, self.dims, x, keep_acts=True)
        val, g = loss(y, tgt, loss_mode, loss_eps)
        G = backward(self.W, self.dims, acts, g)
        self.t += 1
        shampoo_update(self.W, self.m, self.v, self.Ls, self.Rs, self.Ps, G, self.t, self.dims, lr=self.lr,
                       eps_rel=self.eps_rel, interval=self.interval)
        return (val, G) if want_grad else val


# ------------------------------------------------- training-record pipeline --
# The steps around the cache query (Sec. 3.3-3.5, the termination heuristic of
# Sec. 3.4 "Path Termination", Eqs. 3-4), on path vertices laid out as
# synth.make_paths writes them (24 floats per vertex).  Everything is FP64,
# from the definition.  Readings: a vertex's spread term is
# sqrt(|x_{i-1} - x_i|^2 / (pdf_i |cos_i|)); the rendering path ends at the
# first vertex n >= 1 with a(x_1..x_n) > c a_0 (else at the last vertex); a
# training suffix restarts the sum after x_n and ends at the first m > n with
# a(x_n..x_m) > c a_0; an unbiased suffix instead continues from each vertex
# j >= n with probability q (the bounce weighted by 1/q) and ends where the
# roulette stops it.
#
# A termination decision is an integer that floating point decides.  An FP32
# evaluation of a(x_1..x_j) = (sum_i s_i)^2 and of c a_0 is each within a
# relative (2j + 11) u and 10 u of the exact value (u = 2^-24; s_i takes ~5 u,
# the j-term sum j u, the square doubles it; a_0 and the product with c ~10 u),
# so a decision with |a - c a_0| <= TERMINATION_BAND(K) (a + c a_0) may come out
# either way in FP32.  paths_check_decisions accepts such decisions taken the
# other way and nothing else.


def termination_band(K: int) -> float:
    """Relative FP32 band of a termination decision on paths of K vertices."""
    return float((2 * K + 24) * 2.0 ** -24)


def _termination_terms(vtx, camera, c):
    """(s [P,K] spread terms, s[:, 0] = 0; thr [P] = c a_0), FP64 (Eqs. 3-4)."""
    v = np.asarray(vtx, dtype=np.float64)
    x = v[:, :, 0:3]
    cam = np.asarray(camera, dtype=np.float64)
    a0 = np.sum((x[:, 0] - cam[None, :]) ** 2, axis=-1) / (4.0 * math.pi * v[:, 0, 15])
    s = np.zeros(v.shape[:2])
    s[:, 1:] = np.sqrt(np.sum((x[:, :-1] - x[:, 1:]) ** 2, axis=-1) / (v[:, 1:, 14] * v[:, 1:, 15]))
    return s, float(c) * a0


def _suffix_end(s_p, thr_p, n, K):
    """First m > n with (s_{n+1} + .. + s_m)^2 > c a_0, else K - 1."""
    a = 0.0
    for j in range(n + 1, K):
        a += s_p[j]
        if a * a > thr_p:
            return j
    return K - 1


def _roulette_end(vtx_p, n, K, rr_q):
    for j in range(n, K):
        if j == K - 1 or not (vtx_p[j, 22] < np.float32(rr_q)):
            return j
    return K - 1


def _tile_pixels(width, height, tile, ox, oy):
    tiles_x, tiles_y = -(-width // tile), -(-height // tile)
    for t in range(tiles_x * tiles_y):
        ty, tx = divmod(t, tiles_x)
        px, py = tx * tile + ox, ty * tile + oy
        yield t, (py * width + px if px < width and py < height else -1)


def paths_radiance(vtx, n):
    """(render_emitted [P,3], render_throughput [P,3]) of paths ending at
    vertex n[p]: the emitted radiance summed along x_0..x_n with the
    throughput of the bounces before each vertex, and the throughput at x_n."""
    v = np.asarray(vtx, dtype=np.float32)
    P, K, _ = v.shape
    f = v[:, :, 19:22].astype(np.float64)
    le = v[:, :, 16:19].astype(np.float64)
    E = np.zeros((P, 3))
    T = np.ones((P, 3))
    Tn = np.zeros((P, 3))
    for j in range(K):
        live = j <= n
        E[live] += T[live] * le[live, j]
        Tn[j == n] = T[j == n]
        T = T * f[:, j]
    return E, Tn


def paths_terminate(vtx, width: int, height: int, camera, c: float, tile: int, ox: int, oy: int, phase: int,
                    rr_q: float):
    """Returns (n [P], render_emitted [P,3], render_throughput [P,3], tiles) where tiles
    is a list of (pixel, n, m, unbiased) per tile (pixel -1: no training path)."""
    v = np.asarray(vtx, dtype=np.float32)
    P, K, _ = v.shape
    s, thr = _termination_terms(v, camera, c)
    acc = np.cumsum(s, axis=1)
    hit = acc * acc > thr[:, None]
    hit[:, 0] = False
    hit[:, K - 1] = True
    n = np.argmax(hit, axis=1).astype(np.int64)
    E, Tn = paths_radiance(v, n)
    tiles = []
    for t, p in _tile_pixels(width, height, tile, ox, oy):
        if p < 0:
            tiles.append((-1, 0, 0, 0))
            continue
        nn = int(n[p])
        unb = phase >= 0 and t % 16 == phase
        m = _roulette_end(v[p], nn, K, rr_q) if unb else _suffix_end(s[p], thr[p], nn, K)
        tiles.append((p, nn, m, int(unb)))
    return n, E, Tn, tiles


def paths_check_decisions(vtx, width: int, height: int, camera, c: float, tile: int, ox: int, oy: int,
                          phase: int, rr_q: float, n, tiles):
    """Checks decisions taken elsewhere (n [P], tiles [T,4]) against the
    definition: each path end and suffix end must be the FP64 one, or differ
    from it only through decisions within the FP32 band (termination_band).
    Returns (ok, number of paths and suffixes that differ)."""
    v = np.asarray(vtx, dtype=np.float32)
    P, K, _ = v.shape
    s, thr = _termination_terms(v, camera, c)
    band = termination_band(K)
    n = np.asarray(n, dtype=np.int64)

    def valid_end(p, start, end):
        # every decision before `end` may be "no" and the one at `end` "yes" (or end is the last vertex)
        if not (start < end <= K - 1):
            return False
        a = 0.0
        for j in range(start + 1, end + 1):
            a += s[p, j]
            near = abs(a * a - thr[p]) <= band * (a * a + thr[p])
            yes = a * a > thr[p]
            if j < end and yes and not near:
                return False
            if j == end and j < K - 1 and not yes and not near:
                return False
        return True

    ref_n, _, _, ref_tiles = paths_terminate(v, width, height, camera, c, tile, ox, oy, phase, rr_q)
    differ = 0
    for p in range(P):
        if n[p] != ref_n[p]:
            if not valid_end(p, 0, int(n[p])):
                return False, differ
            differ += 1
    tiles = np.asarray(tiles).reshape(-1, 4)
    if len(tiles) != len(ref_tiles):
        return False, differ
    for (p, nn, m, unb), ref in zip(tiles.tolist(), ref_tiles):
        if p != ref[0] or unb != ref[3]:
            return False, differ
        if p < 0:
            continue
        if nn != n[p]:
            return False, differ
        want = _roulette_end(v[p], nn, K, rr_q) if unb else _suffix_end(s[p], thr[p], nn, K)
        if m != want:
            if unb or not valid_end(p, nn, m):
                return False, differ
            differ += 1
    return True, differ


def paths_records(vtx, tiles, tail_rgb, rr_q: float):
    """Training records and self-training targets (Sec. 3.3): for each training
    path (tiles in order) the vertices 0 .. m-1 with the reflected radiance
    transported back from the tail (the cache's value at x_m, or 0 where the
    roulette ended an unbiased suffix).  Returns (records [N,16] float32, targets [N,3])."""
    vtx = np.asarray(vtx, dtype=np.float32)
    recs, tgts = [], []
    for t, (p, n, m, unb) in enumerate(tiles):
        if p < 0:
            continue
        L = np.zeros(3) if unb else np.asarray(tail_rgb[t], dtype=np.float64)
        out = []
        for j in range(m - 1, -1, -1):
            w = vtx[p, j, 19:22].astype(np.float64)
            if unb and j >= n:
                w = w / np.float64(np.float32(rr_q))
            L = w * (vtx[p, j + 1, 16:19].astype(np.float64) + L)
            out.append((j, L.copy()))
        for j, L in reversed(out):
            r = np.zeros(16, dtype=np.float32)
            r[0:14] = vtx[p, j, 0:14]
            recs.append(r)
            tgts.append(L)
    if not recs:
        return np.zeros((0, 16), np.float32), np.zeros((0, 3))
    return np.array(recs, dtype=np.float32), np.array(tgts)


def paths_composite(emitted, throughput, rgb):
    """Pixel radiance: emitted light along the rendering path plus the path
    throughput times the cache's value at its terminal vertex."""
    return np.asarray(emitted, np.float64) + np.asarray(throughput, np.float64) * np.asarray(rgb, np.float64)
