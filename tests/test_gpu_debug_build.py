"""The NRC_DEBUG build (device bounds checks that set the error word instead
of accessing out of range) runs small odd-size cases clean.

Two child processes run the same calls on cuda:0 -- queries of n = 1, 127 and
129 records, a training step of 129 records, a fused frame of 129 queries and
two 129-record steps, for FP16 and FP32 -- one with the ordinary library and
one with libnrc_debug.so (NRC_LIB_VARIANT=debug).  Every call of the debug run
must leave the error word clear (nrc_check_error: NRC_ERR_BOUNDS otherwise),
and the two runs must give the same bits: the checks guard accesses, not
arithmetic.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
from paper_2106_12372_gb300 import build, nrc, synth
build.build()
dev = torch.device("cuda:0")
dims = synth.layer_dims()
w0 = synth.xavier_weights(dims, seed=7)
pool, tgt = (torch.from_numpy(a).to(dev) for a in synth.make_training_pool(1000, seed=3))
out = {"lib": np.frombuffer(nrc.LIB_PATH.encode(), dtype=np.uint8)}
for dtype in ("fp16", "fp32"):
    for n in (1, 127, 129):
        rec = torch.from_numpy(synth.make_records(n, seed=n)).to(dev)
        c = nrc.Cache(dtype=dtype)
        c.set_state(w0)
        out[f"infer_{dtype}_{n}"] = c.infer(rec).cpu().numpy()
        c.check_error()
        c.close()
    c = nrc.Cache(dtype=dtype)
    c.set_state(w0)
    loss = torch.zeros(1, device=dev)
    c.train_step(pool, tgt, 129, synth.frame_seed(3, 0), 0, loss_out=loss)
    c.check_error()
    out[f"train_{dtype}_w"], out[f"train_{dtype}_m"] = c.get_state()[:2]
    out[f"train_{dtype}_loss"] = loss.cpu().numpy()
    q = torch.from_numpy(synth.make_records(129, seed=5)).to(dev)
    rgb = torch.empty((129, 3), device=dev)
    losses = torch.zeros(2, device=dev)
    c.frame(q, rgb, pool, tgt, 129, 2, synth.frame_seed(3, 1), loss_out=losses)
    c.check_error()
    out[f"frame_{dtype}_rgb"], out[f"frame_{dtype}_loss"] = rgb.cpu().numpy(), losses.cpu().numpy()
    out[f"frame_{dtype}_w"] = c.get_state()[0]
    c.close()
np.savez(sys.argv[1], **out)
'''


def _run(variant, path):
    env = dict(os.environ, NRC_LIB_VARIANT=variant, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT, path], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, (r.stdout + r.stderr)[-3000:]
    return np.load(path)


def test_debug_build_runs_odd_sizes_clean_and_identical(tmp_path):
    plain = _run("", str(tmp_path / "plain.npz"))
    debug = _run("debug", str(tmp_path / "debug.npz"))
    assert bytes(debug["lib"]).endswith(b"libnrc_debug.so") and bytes(plain["lib"]).endswith(b"libnrc.so")
    for k in plain.files:
        if k != "lib":
            assert np.array_equal(plain[k].view(np.uint8), debug[k].view(np.uint8)), k
