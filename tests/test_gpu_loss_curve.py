"""1000-step training-loss curves of the CUDA path against the FP64 oracle's
(tests/golden/loss_curve_fp64.json, written by tests/golden/make_loss_curve.py).

Online training with Adam at lr 1e-2 on the relative L2 loss is chaotic: in the
FP64 oracle itself a 1e-7 relative perturbation of the initial weights moves
the 10-step moving average of the loss by 5 % within ~50 steps and the weights
by ~40 % within 300 steps, while the median loss over any 100-step window stays
within ~1-2 %.  So the curves are compared where they are reproducible: step
by step over the first steps, and by the median of every 100-step window
(within 5 %) over all 1000 steps.
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
POINTWISE = {"fp32": (1e-2, 40), "fp16": (5e-2, 10), "bf16": (5e-2, 5)}


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
    failures = []
    for dt, c in caches.items():
        c.check_error()
        got = losses[dt].cpu().numpy().astype(np.float64)
        tol, n_pw = POINTWISE[dt]
        pw = np.abs(got[:n_pw] - ref[:n_pw]) / ref[:n_pw]
        med_ref = np.array([np.median(ref[i:i + 100]) for i in range(0, len(ref), 100)])
        med_got = np.array([np.median(got[i:i + 100]) for i in range(0, len(got), 100)])
        wdev = np.abs(med_got - med_ref) / med_ref
        print(dt, "pointwise max over first", n_pw, pw.max(), "window-median deviations", np.round(wdev, 4),
              "overall median", np.median(got), np.median(ref))
        if pw.max() > tol or wdev.max() > 0.05 or not np.all(np.isfinite(got)):
            failures.append((dt, pw.max(), wdev.max()))
    assert not failures, failures
