"""FP8 E4M3 queries (dtype NRC_FP8) on the GPU.

Two references, both independent of the CUDA path:
* an emulation of the scaled E4M3 arithmetic written here from the format's
  definition (4 exponent bits, bias 7, 3 mantissa bits, subnormals down to
  2^-9, saturation at 448, round to nearest even), with the products in FP64:
  the GPU matches it except where an accumulation-order difference moves a
  value across an E4M3 rounding boundary;
* the FP64 oracle (exact arithmetic): the error of FP8 queries is stated.
Training in an FP8 cache runs in FP16; the FP8 image follows the trained weights.
"""
import numpy as np
import pytest

from paper_2106_12372_gb300 import synth
from parity import rel_err, stats

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2106_12372_gb300 import build, nrc  # noqa: E402

DEV = torch.device("cuda:0")
DIMS = synth.layer_dims()


def e4m3(x):
    """Round to the nearest E4M3 value (ties to even), saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -30)))
    spacing = 2.0 ** (np.maximum(e, -6.0) - 3.0)  # 3 mantissa bits; below 2^-6 the subnormal spacing 2^-9
    q = np.round(a / spacing) * spacing  # numpy rounds halves to even
    return np.sign(x) * np.minimum(q, 448.0)


def pow2_scale(a):
    """2^(7 - floor(log2 a)) (1 for a == 0)."""
    return np.where(a > 0, 2.0 ** (7.0 - np.floor(np.log2(np.maximum(a, 1e-300)))), 1.0)


def emulate(w, rec):
    x = O.encode(rec)  # FP64 features (the kernel rounds its FP32 features; rare boundary differences)
    a = e4m3(128.0 * x)
    inv = np.full(len(rec), 1.0 / 128.0)
    off = 0
    L = len(DIMS) - 1
    for l in range(L):
        W = w[off:off + DIMS[l] * DIMS[l + 1]].reshape(DIMS[l + 1], DIMS[l]).astype(np.float64)
        off += W.size
        s = pow2_scale(np.abs(W).max())
        D = a @ e4m3(W * s).T
        inv = inv / s
        if l + 1 < L:
            c = pow2_scale(np.maximum(D.max(axis=1), 0.0))
            a = e4m3(np.maximum(D, 0.0) * c[:, None])
            inv = inv / c
        else:
            return D * inv[:, None]


def test_e4m3_rounding_definition():
    assert e4m3(448.0) == 448.0 and e4m3(1e6) == 448.0 and e4m3(-500.0) == -448.0
    assert e4m3(2.0 ** -9) == 2.0 ** -9 and e4m3(2.0 ** -11) == 0.0
    assert e4m3(1.0 + 1.0 / 16) == 1.0  # tie between 1 and 1.125 -> even mantissa
    assert e4m3(1.0 + 3.0 / 16) == 1.25  # tie between 1.125 and 1.25 -> even mantissa
    assert e4m3(0.1) == pytest.approx(0.1015625)


@pytest.mark.parametrize("n", [1000, 40_000])
def test_fp8_queries_match_the_e4m3_emulation_and_state_the_error(n):
    build.build()
    w0 = synth.xavier_weights(DIMS, seed=31)
    c = nrc.Cache(dtype="fp8", seed=31)
    c.set_state(w0)
    rec = synth.make_records(n, seed=32)
    got = c.infer(torch.from_numpy(rec).to(DEV)).cpu().numpy()
    emu = emulate(w0, rec)
    e = rel_err(got, emu)
    print("fp8 vs E4M3 emulation", stats(got, emu))
    assert np.median(e) <= 1e-5
    assert np.quantile(e, 0.99) <= 2e-2
    ref = O.infer(w0, DIMS, rec)
    s = stats(got, ref)
    print("fp8 vs FP64 oracle", s)
    # E4M3 keeps 3 mantissa bits (relative rounding up to 6.25 %); measured
    # through the six layers: median 6.5e-2, maximum 0.4-0.6 of the rms
    assert s["median"] <= 0.1
    c.check_error()


def test_fp8_cache_trains_and_queries_follow_the_weights():
    c8 = nrc.Cache(dtype="fp8", seed=41)
    c16 = nrc.Cache(dtype="fp16", seed=41)
    pool, tgt = synth.make_training_pool(4 * 4096, seed=42)
    P, T = torch.from_numpy(pool).to(DEV), torch.from_numpy(tgt).to(DEV)
    for f in range(3):
        for s in range(4):
            c8.train_step(P, T, 4096, synth.frame_seed(43, f), s)
            c16.train_step(P, T, 4096, synth.frame_seed(43, f), s)
    w8, w16 = c8.get_state()[0], c16.get_state()[0]
    assert np.array_equal(w8, w16)  # FP8 caches train exactly as FP16 caches
    rec = synth.make_records(5000, seed=44)
    got = c8.infer(torch.from_numpy(rec).to(DEV)).cpu().numpy()
    assert rel_err(got, emulate(w8, rec)).max() <= 0.1
    assert np.median(rel_err(got, emulate(w8, rec))) <= 1e-5
    with pytest.raises(nrc.NrcError):
        nrc.Batch([c8])
    c8.check_error()
