"""The allocation-free training step (nrc_train_step_noalloc) against the ordinary one.

For callers that cannot allocate device memory when they train (an engine
that owns every device allocation, a frame loop that must not synchronise
the device): the entry point keeps its scratch in fixed-size static device
arrays and trains state the caller owns.  Two calls in a row must give what
nrc_train_step gives on a cache holding the same state, within the 16-bit
path's tolerance, while every library allocation is set to fail and the
device's free memory stays the same (after the start-up call with batch 0,
which loads the module that holds the scratch).  The file's name makes pytest collect
it last.
"""
import numpy as np
import pytest

from paper_2106_12372_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2106_12372_gb300 import build, nrc  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 2e-2  # the FP16 tensor-core path's bound


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), np.sqrt(np.mean(b ** 2)))


def test_noalloc_matches_train_step_twice():
    build.build()
    dims = synth.layer_dims()
    w0 = synth.xavier_weights(dims, seed=321)
    pool_np, tgt_np = synth.make_training_pool(65536, seed=322)
    pool, tgt = torch.from_numpy(pool_np).to(DEV), torch.from_numpy(tgt_np).to(DEV)
    fs = synth.frame_seed(321, 0)

    ref = nrc.Cache(dtype="fp16")
    ref.set_state(w0)
    cfg = nrc.default_config(dtype="fp16")
    w = torch.from_numpy(w0.copy()).to(DEV)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    t = torch.zeros(1, dtype=torch.int64, device=DEV)
    err = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    # the start-up call: loads the static scratch (lazy module loading), launches nothing
    nrc.train_step_noalloc(cfg, w, m, v, t, pool, tgt, 0, fs, 0)
    torch.cuda.synchronize()
    assert t.item() == 0
    for step in range(2):
        l_ref = torch.zeros(1, device=DEV)
        l_na = torch.zeros(1, device=DEV)
        ref.train_step(pool, tgt, 16384, fs, step, loss_out=l_ref)
        torch.cuda.synchronize()
        # the property the entry point exists for: with every device allocation
        # the library could make set to fail, the step still succeeds, and the
        # device's free memory does not change across it
        free0 = torch.cuda.mem_get_info()[0]
        nrc.debug_fail_device_allocs(0, 1000)
        try:
            nrc.train_step_noalloc(cfg, w, m, v, t, pool, tgt, 16384, fs, step, loss_out=l_na, err_out=err)
            torch.cuda.synchronize()
        finally:
            nrc.debug_fail_device_allocs(0, 0)
        assert torch.cuda.mem_get_info()[0] == free0
        rw, rm, rv, rt = ref.get_state()
        assert err.item() == 0 and t.item() == rt == step + 1
        assert abs(l_na.item() - l_ref.item()) <= TOL * abs(l_ref.item())
        assert _rel(m.cpu().numpy(), rm).max() <= TOL
        assert _rel(v.cpu().numpy(), rv).max() <= TOL
        # weights: Adam moves each by about lr; elements whose gradient is tiny may take the other sign
        g = rm.astype(np.float64)
        keep = np.abs(g) > 1e-3 * np.sqrt(np.mean(g ** 2))
        dw = np.abs(w.cpu().numpy() - rw)
        assert dw[keep].max() <= TOL * 1e-2
    ref.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    build.build()
    L = nrc.lib()
    dummy = torch.zeros(16, device=DEV)
    cfg = nrc.default_config(dtype="fp16", hidden_layers=7)
    rc = L.nrc_train_step_noalloc(nrc.ctypes.byref(cfg), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                  dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 1 << 17, 1 << 16, 0, 0,
                                  None, None, nrc._stream(None))
    assert rc == nrc.NRC_ERR_INVALID_ARG and b"hidden_layers" in L.nrc_last_error_string()
    cfg = nrc.default_config(dtype="fp16")
    rc = L.nrc_train_step_noalloc(nrc.ctypes.byref(cfg), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                  dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 1 << 18, 1 << 17, 0, 0,
                                  None, None, nrc._stream(None))
    assert rc == nrc.NRC_ERR_INVALID_ARG and b"maximum" in L.nrc_last_error_string()
    # the constants nrc_create checks: a loss epsilon of 0 would divide by zero in Eq. 5
    cfg = nrc.default_config(dtype="fp16", loss_eps=0.0)
    rc = L.nrc_train_step_noalloc(nrc.ctypes.byref(cfg), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                  dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 4, 4, 0, 0,
                                  None, None, nrc._stream(None))
    assert rc == nrc.NRC_ERR_INVALID_ARG and b"constants" in L.nrc_last_error_string()
