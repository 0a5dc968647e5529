"""Pins the 16-bit rounding emulation and error bounds (tests/error_bounds.py), on CPU.

* the worst-case bound's FP64 values are the oracle's (forward of Sec. 5,
  Eq. 5, the backward pass), and so are the emulation's with no rounding;
* the emulated 16-bit arithmetic (every MMA operand rounded to FP16 or BF16,
  round to nearest even) stays inside the worst-case first-order bound at
  every output and every gradient element, at the initial and at spread-out
  weights, both loss modes;
* the emulated error follows the unit roundoff: BF16's is about 8x FP16's
  (2^-8 / 2^-11);
* the tolerance built from it covers the error at every element, and so does
  an independent realization (FP32 accumulation in numpy's order) at widths
  64 and 128.
"""
import numpy as np
import pytest

import error_bounds as EB
import relu_flips as RF
from oracle import oracle as O
from paper_2106_12372_gb300 import synth

DIMS = synth.layer_dims()


def _case(seed, n=2048, spread=False):
    w = synth.xavier_weights(DIMS, seed=seed).astype(np.float64)
    if spread:
        w = w * np.random.default_rng(seed).uniform(0.5, 2.0, w.size)
        w = w.astype(np.float32).astype(np.float64)
    pool, tgt = synth.make_training_pool(n, seed=seed + 1)
    x = O.encode(pool, 0, 1.0)
    return w, pool, x, tgt.astype(np.float64)


@pytest.mark.parametrize("loss_mode", [O.LOSS_LUMINANCE, O.LOSS_PER_CHANNEL])
def test_fp64_gradient_is_the_oracles_in_both_loss_modes(loss_mode):
    w, pool, x, t = _case(13, n=384)
    y, acts = O.forward(w, DIMS, x, keep_acts=True)
    _, gy = O.loss(y, t, loss_mode)
    ref = O.backward(w, DIMS, acts, gy)
    pc = loss_mode == O.LOSS_PER_CHANNEL
    for g in (EB.grad_bound(w, DIMS, x, t, EB.U["fp16"], per_channel=pc)[0],
              EB.emulate_16bit(w, DIMS, x, t, "fp64", per_channel=pc)[1]):
        assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_fp64_values_are_the_oracles():
    w, pool, x, t = _case(11, n=512)
    y, _, _ = EB.forward_bound(w, DIMS, x, EB.U["fp16"])
    assert np.max(np.abs(y - O.infer(w, DIMS, pool))) <= 1e-12 * max(1.0, np.max(np.abs(y)))
    g, _ = EB.grad_bound(w, DIMS, x, t, EB.U["fp16"])
    ref = RF.batch_grad(w, DIMS, x, t)
    assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("dtype", ["fp16", "bf16"])
@pytest.mark.parametrize("spread", [False, True])
@pytest.mark.parametrize("per_channel", [False, True])
def test_bound_contains_the_emulated_16bit_arithmetic(dtype, spread, per_channel):
    w, pool, x, t = _case(20 + spread + 2 * per_channel, spread=spread)
    u = EB.U[dtype]
    y, ey, _ = EB.forward_bound(w, DIMS, x, u)
    g, eg = EB.grad_bound(w, DIMS, x, t, u, per_channel=per_channel)
    y16, g16 = EB.emulate_16bit(w, DIMS, x, t, dtype, per_channel=per_channel)
    err_y, err_g = np.abs(y16 - y), np.abs(g16 - g)
    assert np.all(err_y <= ey), float(np.max(err_y / ey))
    assert np.all(err_g <= eg), float(np.max(err_g / eg))
    print(dtype, "spread" if spread else "init", "per-channel" if per_channel else "luminance",
          "median err/bound: outputs", float(np.median(err_y / ey)), "gradient", float(np.median(err_g / eg)))


def test_emulation_without_rounding_is_the_oracle():
    w, pool, x, t = _case(12, n=512)
    y, g = EB.emulate_16bit(w, DIMS, x, t, "fp64")
    ref_y = O.infer(w, DIMS, pool)
    assert np.max(np.abs(y - ref_y)) <= 1e-12 * np.max(np.abs(ref_y))
    assert np.max(np.abs(EB.emulate_infer(w, DIMS, x, "fp64") - ref_y)) <= 1e-12 * np.max(np.abs(ref_y))
    ref_g = RF.batch_grad(w, DIMS, x, t)
    assert np.max(np.abs(g - ref_g)) <= 1e-12 * np.max(np.abs(ref_g))
    assert np.array_equal(EB.emulate_infer(w, DIMS, x, "fp16"), EB.emulate_16bit(w, DIMS, x, t, "fp16")[0])


def _rms(a):
    return float(np.sqrt(np.mean(np.asarray(a) ** 2)))


def test_emulated_error_follows_the_unit_roundoff():
    w, pool, x, t = _case(31, n=2048)
    y0, g0 = EB.emulate_16bit(w, DIMS, x, t, "fp64")
    y16, g16 = EB.emulate_16bit(w, DIMS, x, t, "fp16")
    y8, g8 = EB.emulate_16bit(w, DIMS, x, t, "bf16")
    ry, rg = _rms(y8 - y0) / _rms(y16 - y0), _rms(g8 - g0) / _rms(g16 - g0)
    print("bf16 / fp16 emulated error rms: outputs", ry, "gradient", rg)
    assert 5.0 <= ry <= 12.0 and 5.0 <= rg <= 12.0, (ry, rg)


@pytest.mark.parametrize("dtype", ["fp16", "bf16"])
@pytest.mark.parametrize("width,hidden", [(64, 5), (128, 7)])
def test_an_fp32_accumulated_realization_stays_inside_the_tolerance(dtype, width, hidden):
    """The GPU sums in FP32 in its own order; numpy's FP32 matrix product does
    too, in another: its result is an independent realization of the rounding
    that the tolerance built from the exact-sum emulation must contain."""
    dims = synth.layer_dims(width=width, hidden_layers=hidden)
    w = synth.xavier_weights(dims, seed=45).astype(np.float64)
    rec = synth.make_records(20000, seed=46)
    x = O.encode(rec)
    ref = EB.emulate_infer(w, dims, x, "fp64")
    e = EB.emulate_infer(w, dims, x, dtype) - ref
    alt = EB.emulate_infer(w, dims, x, dtype, acc32=True) - ref
    ratio = float(np.max(np.abs(alt) / EB.format_tol(e)))
    dev = np.abs(alt - e) / np.sqrt(np.mean(e ** 2))
    print(dtype, width, "worst |alt| / tol", ratio, "rows re-rounded (|alt - e| > rms(e)/10):",
          float(np.mean(dev.max(axis=1) > 0.1)), "max |alt - e| / rms(e)", float(dev.max()))
    assert ratio <= 1.0
    assert np.sqrt(np.mean(alt ** 2)) <= 1.2 * np.sqrt(np.mean(e ** 2))


def test_tail_factor():
    # 1e-6 two-sided tail bound by the union bound: c_1 = sqrt(2 ln 2e6) = 5.39; grows like sqrt(2 ln N)
    assert abs(EB.tail_factor(1) - np.sqrt(2 * np.log(2e6))) < 1e-12
    assert 7.0 < EB.tail_factor(120_000) < 7.5
    from scipy.stats import norm
    n = 1000
    assert 2 * n * norm.sf(EB.tail_factor(n)) <= 1e-6 + 1e-12


@pytest.mark.parametrize("dtype", ["fp16", "bf16"])
def test_format_tolerance_covers_the_emulated_error(dtype):
    w, pool, x, t = _case(41, n=1024)
    y0, g0 = EB.emulate_16bit(w, DIMS, x, t, "fp64")
    y, g = EB.emulate_16bit(w, DIMS, x, t, dtype)
    ty, tg = EB.format_tol(y - y0), EB.format_tol(g - g0, DIMS)
    assert np.all(np.abs(y - y0) <= ty) and np.all(np.abs(g - g0) <= tg)
    # per weight matrix: the rms term is c_N rms of that matrix's error, N its size
    n0 = DIMS[0] * DIMS[1]
    e0 = np.abs(g - g0)[:n0]
    assert np.allclose(tg[:n0], 2 * e0 + EB.tail_factor(n0) * _rms(e0))


def test_bf16_rounding_is_nearest_even():
    # 1 + 2^-8 is the tie between 1 and 1 + 2^-7: even mantissa (1) wins;
    # 1 + 3 * 2^-8 ties between 1 + 2^-7 and 1 + 2^-6... its even neighbour is 1 + 2^-6
    v = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -(1.0 + 2.0 ** -7)])
    assert list(EB.round16(v, "bf16")) == [1.0, 1.0 + 2.0 ** -6, 1.0, -(1.0 + 2.0 ** -7)]
    assert EB.round16(np.array([1.0 + 2.0 ** -11]), "fp16")[0] == 1.0
