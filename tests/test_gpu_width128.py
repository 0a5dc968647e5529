"""The width-128, 7-hidden-layer network (the precision sweep's wide variant)
against the FP64 oracle.  Plain per-layer FP32 path: Xavier weights
bit-identical, queries and one training step within 1e-5, and a 100-step loss
curve that follows the oracle's pointwise over its first steps.  FP16 / BF16
queries on the tensor cores (k_tc128, Sec. 4 / Fig. 5 at width 128): 2e-2 per
output (FP16) and the format tolerance of tests/error_bounds.py (both), at
ragged sizes, both encodings and pad values, and after training steps (which
run on the plain FP32 kernels and keep the 16-bit image current)."""
import json
import os

import numpy as np
import pytest

from paper_2106_12372_gb300 import synth
from parity import rel_err, stats
import error_bounds as EB

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2106_12372_gb300 import build, nrc  # noqa: E402

DEV = torch.device("cuda:0")
DIMS = synth.layer_dims(width=128, hidden_layers=7)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _cache(seed):
    return nrc.Cache(dtype="fp32", path=nrc.PATH_PLAIN, width=128, hidden_layers=7, seed=seed)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_init_and_queries():
    c = _cache(51)
    w = c.get_state()[0]
    assert np.array_equal(w, synth.xavier_weights(DIMS, seed=51))
    rec = synth.make_records(3001, seed=52)
    got = c.infer(dev(rec)).cpu().numpy()
    ref = O.infer(w, DIMS, rec)
    print("width 128 query", stats(got, ref))
    assert rel_err(got, ref).max() <= 1e-5
    c.check_error()


def test_training_step():
    c = _cache(53)
    w0 = c.get_state()[0]
    pool, tgt = synth.make_training_pool(8192, seed=54)
    loss = torch.zeros(1, device=DEV)
    c.train_step(dev(pool), dev(tgt), 4096, synth.frame_seed(55, 0), 1, loss_out=loss)
    st = O.TrainState(w0, DIMS)
    ref_loss, ref_g = st.step(pool, tgt, 4096, synth.frame_seed(55, 0), 1, want_grad=True)
    g = c.get_state()[1].astype(np.float64) / (1.0 - 0.9)
    print("width 128 step", loss.item(), ref_loss, stats(g, ref_g))
    assert abs(loss.item() - ref_loss) <= 1e-5 * abs(ref_loss)
    assert rel_err(g, ref_g).max() <= 1e-5


def test_loss_curve_follows_the_oracle():
    c = _cache(56)
    st = O.TrainState(c.get_state()[0], DIMS)
    pool, tgt = synth.make_training_pool(4 * 2048, seed=57)
    P, T = dev(pool), dev(tgt)
    losses = torch.zeros(100, device=DEV)
    ref = []
    for f in range(25):
        c.frame(P[:0], P[:0], P, T, 2048, 4, synth.frame_seed(58, f), loss_out=losses[4 * f:4 * f + 4])
        for s in range(4):
            ref.append(st.step(pool, tgt, 2048, synth.frame_seed(58, f), s))
    got = losses.cpu().numpy().astype(np.float64)
    ref = np.array(ref)
    print("width 128 curve: first 5", got[:5], ref[:5], "100-step medians", np.median(got), np.median(ref))
    # online training is chaotic: FP32 and FP64 runs agree step by step only at
    # first; afterwards even FP64 runs whose initial weights differ by 1e-7
    # drift apart (tests/golden/width128_curve_fp64.json: 100-step medians up to
    # 17 % apart), so the GPU run's median is held to 1.5 x that spread around
    # the oracle's (the loss-curve reading)
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "width128_curve_fp64.json")))
    spread = max(abs(m - gold["medians"][0]) for m in gold["medians"][1:]) / gold["medians"][0]
    print("oracle realizations' 100-step median spread", spread)
    assert np.all(np.abs(got[:20] - ref[:20]) <= 1e-2 * np.abs(ref[:20]))
    assert abs(np.median(got) - np.median(ref)) <= max(0.05, 1.5 * spread) * np.median(ref)
    c.check_error()


def _format_check(got, ref, emul, label, model_check=True):
    EB.format_check(got, ref, emul, label="width 128 " + label, model_check=model_check)


@pytest.mark.parametrize("dtype", ["fp16", "bf16"])
@pytest.mark.parametrize("n", [1, 127, 129, 4097, 40_000])
def test_tensor_core_queries(dtype, n):
    c = nrc.Cache(dtype=dtype, width=128, hidden_layers=7, seed=61)
    w = c.get_state()[0]
    rec = synth.make_records(n, seed=62 + n)
    got = c.infer(dev(rec)).cpu().numpy()
    ref = O.infer(w, DIMS, rec)
    st = stats(got, ref)
    print("width 128 tensor-core query", dtype, n, st)
    # FP16 meets 2e-2 at every output; BF16 (8 significant bits) misses it at single outputs as at width 64
    # and is held to its format tolerance
    if dtype == "fp16":
        assert st["max"] <= 2e-2, st
    print("99th percentile", float(np.quantile(rel_err(got, ref), 0.99)))
    if n >= 127 and dtype == "fp16":
        assert np.quantile(rel_err(got, ref), 0.99) <= 2e-2
    _format_check(got, ref, EB.emulate_infer(w, DIMS, O.encode(rec), dtype), f"{dtype} {n}", model_check=n >= 127)
    c.check_error()


@pytest.mark.parametrize("mode,pad", [(1, 1.0), (0, 0.0)])
def test_tensor_core_queries_modes(mode, pad):
    c = nrc.Cache(dtype="fp16", width=128, hidden_layers=7, seed=63, enc_mode=mode, pad_value=pad)
    w = c.get_state()[0]
    rec = synth.make_records(3000, seed=64)
    got = c.infer(dev(rec)).cpu().numpy()
    ref = O.infer(w, DIMS, rec, mode, pad)
    assert rel_err(got, ref).max() <= 2e-2
    _format_check(got, ref, EB.emulate_infer(w, DIMS, O.encode(rec, mode, pad), "fp16"), f"mode {mode} pad {pad}")


def test_tensor_core_queries_follow_training():
    # training runs on the plain FP32 kernels; their Adam writes the 16-bit image (blocks of 64 inputs)
    c = nrc.Cache(dtype="fp16", width=128, hidden_layers=7, seed=65)
    pool, tgt = synth.make_training_pool(8192, seed=66)
    P, T = dev(pool), dev(tgt)
    for s in range(3):
        c.train_step(P, T, 2048, synth.frame_seed(67, 0), s)
    w = c.get_state()[0]
    assert not np.array_equal(w, synth.xavier_weights(DIMS, seed=65))
    rec = synth.make_records(5000, seed=68)
    got = c.infer(dev(rec)).cpu().numpy()
    ref = O.infer(w, DIMS, rec)
    assert rel_err(got, ref).max() <= 2e-2
    _format_check(got, ref, EB.emulate_infer(w, DIMS, O.encode(rec), "fp16"), "after 3 steps")
    # a frame (queries on the tensor cores, then the steps) equals the two calls
    q = dev(synth.make_records(1000, seed=69))
    rgb = torch.empty((1000, 3), device=DEV)
    c2 = nrc.Cache(dtype="fp16", width=128, hidden_layers=7, seed=65)
    for s in range(3):
        c2.train_step(P, T, 2048, synth.frame_seed(67, 0), s)
    c.frame(q, rgb, P, T, 2048, 2, synth.frame_seed(67, 1))
    ref_rgb = c2.infer(q)
    c2.train_step(P, T, 2048, synth.frame_seed(67, 1), 0)
    c2.train_step(P, T, 2048, synth.frame_seed(67, 1), 1)
    assert torch.equal(rgb, ref_rgb)
    assert np.array_equal(c.get_state()[0], c2.get_state()[0])
    c.check_error()


def test_width128_rejections():
    # FP32 stays on the plain path; the tensor cores take at most 7 hidden layers, no weight average, Adam only
    c = _cache(59)
    with pytest.raises(nrc.NrcError):
        c.set_path(nrc.PATH_FUSED)
    for kw in ({"dtype": "fp32"}, {"dtype": "fp16", "hidden_layers": 8}, {"dtype": "fp16", "ema": 1},
               {"dtype": "fp8"}):
        args = dict(width=128, hidden_layers=7)
        args.update(kw)
        with pytest.raises(nrc.NrcError):
            nrc.Cache(**args)
    # the batched caches take the width-64 network only
    with pytest.raises(nrc.NrcError):
        nrc.Batch([nrc.Cache(dtype="fp16", width=128, hidden_layers=7)])
