"""The width-128, 7-hidden-layer network on the plain per-layer FP32 path
(the precision sweep's wide variant) against the FP64 oracle: Xavier weights
bit-identical, queries and one training step within 1e-5, and a 100-step loss
curve that follows the oracle's pointwise over its first steps."""
import json
import os

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


def test_fused_paths_take_width_64_only():
    with pytest.raises(nrc.NrcError):
        nrc.Cache(dtype="fp16", width=128, hidden_layers=7)
    c = _cache(59)
    with pytest.raises(nrc.NrcError):
        c.set_path(nrc.PATH_FUSED)
