"""ReLU decisions that FP32 and FP64 may take differently (test helper).

A ReLU mask is an integer that floating point decides.  A pre-activation that
lies within the FP32 rounding of a 64-term dot product of zero may come out
positive in one precision and negative in the other, and then one record's
delta for that unit is in one gradient and not in the other: a whole row of
that layer's weight gradient moves by that record's contribution (up to ~3e-4
relative on a 16,384-record batch).  Both results are correct to their
precision.  This module finds such decisions in an FP64 forward pass and
computes, for each, the exact change of the batch gradient if that one
decision were taken the other way; `explain` removes from a GPU-minus-oracle
difference the changes that reduce it, so that a test can hold what is left
to the FP32 tolerance.

The arithmetic (forward, relative-L2 loss of Eq. 5 with the luminance
denominator, backward) is an FP64 numpy restatement used only for this;
`tests/test_oracle_relu_flips.py` pins its gradient to the oracle's.
"""
import numpy as np

LUM = np.array([0.2126, 0.7152, 0.0722])


def _mats(w, dims):
    out, off = [], 0
    for l in range(len(dims) - 1):
        n = dims[l] * dims[l + 1]
        out.append(np.asarray(w[off:off + n], dtype=np.float64).reshape(dims[l + 1], dims[l]))
        off += n
    return out


def _grad_rows(Ws, x, t, n_total, loss_eps, flip=None):
    """Gradient (flat) of the mean loss over n_total records, contributed by rows x."""
    H, masks, h = [x], [], x
    for l, W in enumerate(Ws):
        z = h @ W.T
        if l + 1 < len(Ws):
            m = z > 0
            if flip is not None and flip[0] == l:
                m[flip[1], flip[2]] = ~m[flip[1], flip[2]]
            masks.append(m)
            h = z * m
        else:
            h = z
        H.append(h)
    y = H[-1]
    lum = y @ LUM
    d = 2.0 * (y - t) / (lum * lum + loss_eps)[:, None] / (3.0 * n_total)
    G = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        G[l] = (d.T @ H[l]).ravel()
        if l > 0:
            d = (d @ Ws[l]) * masks[l - 1]
    return np.concatenate(G)


def batch_grad(w, dims, x, t, loss_eps=0.01):
    """FP64 gradient of the batch's mean relative-L2 loss (luminance denominator)."""
    return _grad_rows(_mats(w, dims), np.asarray(x, np.float64), np.asarray(t, np.float64), len(x), loss_eps)


def ambiguous_flips(w, dims, x, t, band=8e-6, loss_eps=0.01):
    """[(layer, row, unit, delta_g)] for every hidden pre-activation z with
    |z| <= band * sum_k |w_k h_k|; delta_g is the change of the batch gradient
    when that decision alone is taken the other way."""
    Ws = _mats(w, dims)
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    out, h = [], x
    cand = []
    for l, W in enumerate(Ws[:-1]):
        z = h @ W.T
        s = np.abs(h) @ np.abs(W).T
        for r, u in np.argwhere(np.abs(z) <= band * s):
            cand.append((l, int(r), int(u)))
        h = np.maximum(z, 0.0)
    for l, r, u in cand:
        base = _grad_rows(Ws, x[r:r + 1], t[r:r + 1], len(x), loss_eps)
        flip = _grad_rows(Ws, x[r:r + 1], t[r:r + 1], len(x), loss_eps, flip=(l, 0, u))
        out.append((l, r, u, flip - base))
    return out


def explain(got, ref, flips):
    """The oracle gradient with those of `flips` taken the other way that make
    it closer to `got` (greedy, largest change first); returns (adjusted ref,
    number of decisions used)."""
    got = np.asarray(got, np.float64)
    adj = np.asarray(ref, np.float64).copy()
    used = 0
    for _, _, _, dg in sorted(flips, key=lambda f: -float(np.linalg.norm(f[3]))):
        if np.linalg.norm(got - adj - dg) < np.linalg.norm(got - adj):
            adj += dg
            used += 1
    return adj, used
