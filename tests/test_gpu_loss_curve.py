"""1000-step training-loss curves of the CUDA path against the FP64 oracle's
(tests/golden/loss_curve_fp64.json, written by tests/golden/make_loss_curve.py).

Online training with Adam at lr 1e-2 on the relative L2 loss is chaotic: two
runs of the FP64 oracle whose initial weights differ by 1e-7 (relative) drift
apart -- their per-step losses differ by up to 0.9 % within 40 steps, the
medians of their 100-step windows by up to 7 % (golden realizations r1, r2),
while the median loss over all 1000 steps stays within ~1 %.  So the curves
are compared where a faithful implementation can be held to them:
* step by step over the leading steps;
* the median loss over the 1000 steps within 5 % of the oracle's;
* each 100-step window median within the oracle realizations' own spread
  (the largest window deviation between them, with a 1.5x margin, and never
  tighter than 5 %).
"""
import json
import os

import numpy as np
import pytest

from paper_2106_12372_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2106_12372_gb300 import build, nrc  # noqa: E402

DEV = torch.device("cuda:0")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "loss_curve_fp64.json")
# pointwise bound and the number of leading steps it applies to, per dtype
POINTWISE = {"fp32": (1e-2, 20), "fp16": (5e-2, 10), "bf16": (5e-2, 5)}


def window_medians(x, w=100):
    return np.array([np.median(x[i:i + w]) for i in range(0, len(x), w)])


def test_loss_curves_track_the_oracle():
    build.build()
    spec = json.load(open(GOLDEN))
    seed, frames, steps, batch = spec["seed"], spec["frames"], spec["steps_per_frame"], spec["batch"]
    ref = np.array(spec["loss"])
    dims = synth.layer_dims()
    w0 = synth.xavier_weights(dims, seed=seed)
    caches = {}
    for dt in POINTWISE:
        caches[dt] = nrc.Cache(dtype=dt)
        caches[dt].set_state(w0)
    losses = {dt: torch.zeros(frames * steps, device=DEV) for dt in POINTWISE}
    for f in range(frames):
        pool_np, tgt_np = synth.make_training_pool(batch * steps, seed=seed * 1000 + f)
        pool, tgt = torch.from_numpy(pool_np).to(DEV), torch.from_numpy(tgt_np).to(DEV)
        fs = synth.frame_seed(seed, f)
        for dt, c in caches.items():
            for s in range(steps):
                k = f * steps + s
                c.train_step(pool, tgt, batch, fs, s, loss_out=losses[dt][k:k + 1])
    torch.cuda.synchronize()
    others = [np.array(json.load(open(GOLDEN.replace(".json", f"_r{k}.json")))["loss"]) for k in (1, 2)]
    wref = window_medians(ref)
    spread = max(np.max(np.abs(window_medians(o) - wref) / wref) for o in others)
    wtol = max(0.05, 1.5 * spread)
    failures = []
    for dt, c in caches.items():
        c.check_error()
        got = losses[dt].cpu().numpy().astype(np.float64)
        tol, n_pw = POINTWISE[dt]
        pw = np.abs(got[:n_pw] - ref[:n_pw]) / ref[:n_pw]
        wdev = np.abs(window_medians(got) - wref) / wref
        mdev = abs(np.median(got) - np.median(ref)) / np.median(ref)
        print(dt, "pointwise max over first", n_pw, pw.max(), "overall-median deviation", mdev,
              "window-median deviations", np.round(wdev, 4), "window tolerance", wtol)
        if pw.max() > tol or mdev > 0.05 or wdev.max() > wtol or not np.all(np.isfinite(got)):
            failures.append((dt, pw.max(), mdev, wdev.max()))
    assert not failures, failures
