"""Process-wide launch state: a kernel's dynamic shared-memory limit is raised
when a later cache needs more than an earlier one (checked in a fresh process,
so that no earlier test has set it already): an FP32 cache of 1 hidden layer
(17 KB of weights in shared memory), then one of 5 (83 KB), then FP16 caches of
both depths, all query and train."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import torch
from paper_2106_12372_gb300 import build, nrc, synth
build.build()
dev = torch.device("cuda:0")
rec = torch.from_numpy(synth.make_records(3000, seed=1)).to(dev)
pool, tgt = (torch.from_numpy(x).to(dev) for x in synth.make_training_pool(4096, seed=2))
for dtype in ("fp32", "fp16"):
    for layers in (1, 5):
        c = nrc.Cache(dtype=dtype, hidden_layers=layers, seed=3)
        y = c.infer(rec)
        c.train_step(pool, tgt, 1024, synth.frame_seed(4, 0), 0)
        c.check_error()
        assert torch.isfinite(y).all()
print("ok")
"""


def test_smem_limit_grows_with_later_caches():
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.stdout[-2000:], r.stderr[-2000:])
