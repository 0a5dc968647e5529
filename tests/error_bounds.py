"""Running error bounds of the 16-bit tensor-core path (test helper).

The 16-bit path rounds every MMA operand (encoded inputs, weights,
activations, deltas) to FP16 or BF16, unit roundoff u = 2^-11 or 2^-8, and
accumulates in FP32.  To first order in u, with |.| taken elementwise and
every quantity the FP64 value of the FP64 forward / backward pass:

  forward   E_H0 = u |H0|
            E_Z  = E_H |W|^T + u |H| |W|^T          (operands rounded)
            E_H' = E_Z + u |H'|                      (ReLU is 1-Lipschitz; result rounded)
            E_y  = E_H |W_L|^T + u |H| |W_L|^T
  loss      g = 2 (y - t) / den of Eq. 5: E_g from dg/dy and dg/dden (den taken
            at its lower end), plus u |g| (the delta is rounded)
  backward  E_P  = E_d |W| + u |d| |W|               (pre-mask delta)
            E_d' = m E_P + u |d'|, and |P| + E_P where the ReLU decision is
                   within the forward bound of zero (it may go either way)
  gradient  E_G  = E_d^T |H| + |d|^T E_H + E_d^T E_H
plus the FP32 accumulation (64-term sums: 64 * 2^-24 of the magnitude sum).
This worst-case bound is sound but loose: it takes every rounding error with
the sign that adds up, so it grows by the row sums of |W| (about 7 at the
initial weights) per layer while the actual errors largely cancel.  It pins
the emulation below (every emulated error lies inside it) and is not used as
a tolerance.

The tolerance of the 16-bit parity tests comes from `emulate_16bit`: the
oracle's arithmetic with exactly the operand roundings of the 16-bit format
(every MMA operand rounded to nearest even; sums exact), so e = emulated -
FP64 is the error the format alone causes.  The GPU additionally sums in
FP32 in its own order: in about 1 % of the rows that rounds an activation to
the neighbouring 16-bit value, which shifts every later pre-activation of the
row by a 16-bit ulp, so that the later roundings go either way and the row's
result is another realization of the format's rounding error, of the same
size as e but not equal to it.  `format_tol` covers that: per element
2 |e_i| + c_N rms(e), c_N = sqrt(2 ln(2 N / 1e-6)) the bound that N normal
draws of standard deviation rms(e) stay within with probability 1 - 1e-6
(rms and N per weight matrix for gradients).  `tests/test_error_bounds.py`
pins the emulation (no rounding gives the oracle; its error follows the unit
roundoff; it lies inside the worst-case bound) and the tolerance (an
independent realization -- the same arithmetic with FP32 accumulation in
numpy's order -- stays inside it at every element).  The arithmetic
restates the network of Sec. 5 in FP64 numpy for this purpose only.
"""
import numpy as np

LUM = np.array([0.2126, 0.7152, 0.0722])
U = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
GAMMA32 = 64 * 2.0 ** -24  # FP32 accumulation of a 64-term sum, relative to the magnitude sum


def _mats(w, dims):
    out, off = [], 0
    for l in range(len(dims) - 1):
        n = dims[l] * dims[l + 1]
        out.append(np.asarray(w[off:off + n], dtype=np.float64).reshape(dims[l + 1], dims[l]))
        off += n
    return out


def forward_bound(w, dims, x, u):
    """(y, E_y, acts): FP64 outputs, their error bound, and the forward state."""
    Ws = _mats(w, dims)
    h = np.asarray(x, np.float64)
    eh = u * np.abs(h) + 2e-7  # the FP32 encoding before the rounding
    H, EH, Z, EZ = [h], [eh], [], []
    for l, W in enumerate(Ws):
        A = np.abs(W)
        z = h @ W.T
        ez = eh @ A.T + (u + GAMMA32) * (np.abs(h) @ A.T)
        Z.append(z)
        EZ.append(ez)
        if l + 1 < len(Ws):
            h = np.maximum(z, 0.0)
            eh = ez + u * np.abs(h)
            H.append(h)
            EH.append(eh)
    return Z[-1], EZ[-1], (Ws, H, EH, Z, EZ)


def grad_bound(w, dims, x, t, u, loss_eps=0.01, per_channel=False):
    """(g, E_g): the FP64 gradient of the batch's mean relative-L2 loss (flat,
    layer after layer, row-major [out][in]) and its elementwise error bound."""
    y, ey, (Ws, H, EH, Z, EZ) = forward_bound(w, dims, x, u)
    t = np.asarray(t, np.float64)
    n = len(t)
    if per_channel:
        den = y * y + loss_eps
        den_lo = np.maximum(np.abs(y) - ey, 0.0) ** 2 + loss_eps
        g = 2.0 * (y - t) / den
        eg = (2.0 / den_lo + 4.0 * (np.abs(y - t) + ey) * (np.abs(y) + ey) / den_lo ** 2) * ey
    else:
        lum = y @ LUM
        elum = ey @ LUM
        den = lum * lum + loss_eps
        den_lo = np.maximum(np.abs(lum) - elum, 0.0) ** 2 + loss_eps
        g = 2.0 * (y - t) / den[:, None]
        eg = 2.0 * ey / den_lo[:, None] + (4.0 * (np.abs(y - t) + ey) * ((np.abs(lum) + elum) * elum)[:, None]
                                            / (den_lo ** 2)[:, None])
    eg = eg + u * np.abs(g)
    d, ed = g, eg
    G, EG = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        h, eh = H[l], EH[l]
        G[l] = d.T @ h
        EG[l] = ed.T @ np.abs(h) + np.abs(d).T @ eh + ed.T @ eh + GAMMA32 * (np.abs(d).T @ np.abs(h))
        if l > 0:
            A = np.abs(Ws[l])
            p = d @ Ws[l]
            ep = ed @ A + (u + GAMMA32) * (np.abs(d) @ A)
            m = Z[l - 1] > 0
            amb = np.abs(Z[l - 1]) <= EZ[l - 1]
            d = p * m
            ed = np.where(amb, np.abs(p) + ep, m * ep) + u * np.abs(d)
    scale = 1.0 / (3.0 * n)
    return np.concatenate([gl.ravel() for gl in G]) * scale, np.concatenate([e.ravel() for e in EG]) * scale


def round16(a, dtype):
    """Round to FP16 or BF16 (nearest even), returned as FP64; "fp64" leaves it."""
    a = np.asarray(a, np.float64)
    if dtype == "fp64":  # no rounding: the emulation is then the FP64 pass
        return a
    if dtype == "fp16":
        return a.astype(np.float16).astype(np.float64)
    b = a.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def emulate_16bit(w, dims, x, t, dtype, loss_eps=0.01, per_channel=False):
    """(y, g): the 16-bit path's arithmetic emulated exactly (operands rounded,
    sums in FP64 -- the FP32 accumulation is the bound's GAMMA32 term)."""
    Ws = [round16(W, dtype) for W in _mats(w, dims)]
    h = round16(x, dtype)
    H, M = [h], []
    for l, W in enumerate(Ws):
        z = h @ W.T
        if l + 1 < len(Ws):
            h = round16(np.maximum(z, 0.0), dtype)
            M.append(h > 0)
            H.append(h)
    y = z
    t = np.asarray(t, np.float64)
    if per_channel:
        g = 2.0 * (y - t) / (y * y + loss_eps)
    else:
        lum = y @ LUM
        g = 2.0 * (y - t) / (lum * lum + loss_eps)[:, None]
    d = round16(g, dtype)
    G = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        G[l] = d.T @ H[l]
        if l > 0:
            d = round16((d @ Ws[l]) * M[l - 1], dtype)
    return y, np.concatenate([gl.ravel() for gl in G]) / (3.0 * len(t))


def emulate_infer(w, dims, x, dtype, acc32=False):
    """Outputs of the 16-bit query path (operands rounded; sums exact, or with
    acc32 in FP32 in numpy's order: another realization of the rounding)."""
    Ws = [round16(W, dtype) for W in _mats(w, dims)]
    h = round16(x, dtype)
    for l, W in enumerate(Ws):
        if acc32:
            z = (h.astype(np.float32) @ W.T.astype(np.float32)).astype(np.float64)
        else:
            z = h @ W.T
        if l + 1 < len(Ws):
            h = round16(np.maximum(z, 0.0), dtype)
    return z


def tail_factor(n, delta=1e-6):
    """c_N: n normal draws of unit standard deviation all lie within +-c_N
    with probability >= 1 - delta (union bound on the normal tail)."""
    return float(np.sqrt(2.0 * np.log(2.0 * max(int(n), 1) / delta)))


def format_tol(err, dims=None):
    """Per-element tolerance 2 |e| + c_N rms(e) of an emulated error e; with
    dims, e is a flat gradient and the rms and N are taken per weight matrix."""
    err = np.abs(np.asarray(err, np.float64))
    if dims is None:
        return 2.0 * err + tail_factor(err.size) * np.sqrt(np.mean(err ** 2))
    out, off = np.empty_like(err), 0
    for l in range(len(dims) - 1):
        n = dims[l] * dims[l + 1]
        e = err[off:off + n]
        out[off:off + n] = 2.0 * e + tail_factor(n) * np.sqrt(np.mean(e ** 2))
        off += n
    return out


def format_check(got, ref, emul, dims=None, label="", model_check=True):
    """Asserts |got - ref| <= format_tol(emul - ref) at every element and, with
    model_check, rms(got - emul) <= rms(emul - ref) / 2; returns the worst
    ratio to the tolerance and that rms ratio."""
    got, ref, emul = (np.asarray(a, np.float64).ravel() for a in (got, ref, emul))
    e = emul - ref
    worst = float(np.max(np.abs(got - ref) / format_tol(e, dims)))
    model = float(np.sqrt(np.mean((got - emul) ** 2)) / np.sqrt(np.mean(e ** 2)))
    print("format bound", label, "max |err| / tol", worst, "rms(gpu - rounding) / rms(rounding error)", model)
    assert worst <= 1.0, (label, worst)
    if model_check:
        assert model <= 0.5, (label, model)
    return worst, model
