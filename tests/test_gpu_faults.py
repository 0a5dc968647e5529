"""Failure detection with faults made on the host (nothing here faults, traps
or hangs the GPU):

* a bounded device wait -- the same wait the kernels use on their mbarriers --
  on an mbarrier nothing arrives at gives up after its limit; the cache reports
  NRC_ERR_TIMEOUT once and keeps answering queries with the same results;
* injected device-allocation failures at every allocation of nrc_create, of a
  cache's first training step, of the batched-cache plan and of a server
  viewport return NRC_ERR_OOM and leave no device memory behind;
* (admission over the memory budget is NRC_ERR_BUSY: test_gpu_serve.py).
"""
import time

import pytest

from paper_2106_12372_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2106_12372_gb300 import build, nrc  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    yield
    nrc.debug_fail_device_allocs(0, 0)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_bounded_wait_times_out_and_the_cache_recovers():
    c = nrc.Cache(dtype="fp16", seed=3)
    rec = torch.from_numpy(synth.make_records(1000, seed=4)).to(DEV)
    ref = c.infer(rec).clone()
    c.check_error()
    t0 = time.perf_counter()
    c.debug_wait_timeout(20_000)  # 20 ms
    with pytest.raises(nrc.NrcError) as ei:
        c.check_error()
    dt = time.perf_counter() - t0
    assert ei.value.status == nrc.NRC_ERR_TIMEOUT
    assert 0.015 <= dt < 2.0, dt
    c.check_error()  # reported once: the word was cleared
    assert torch.equal(c.infer(rec), ref)
    c.check_error()


def _fail_each(make, max_allocs=40):
    """Fails allocation k of make() for k = 0, 1, ... until make() succeeds;
    returns the number of allocations it needed."""
    for after in range(max_allocs):
        nrc.debug_fail_device_allocs(after, 1)
        try:
            obj = make()
        except nrc.NrcError as e:
            assert e.status == nrc.NRC_ERR_OOM, (after, e)
            continue
        finally:
            nrc.debug_fail_device_allocs(0, 0)
        return after, obj
    raise AssertionError("never succeeded")


def test_allocation_failures_in_create_report_oom_and_leak_nothing():
    nrc.Cache(dtype="fp16").close()  # lazily created library state
    before = _free_bytes()
    n, c = _fail_each(lambda: nrc.Cache(dtype="fp16", ema=True, optimizer=nrc.OPT_SHAMPOO))
    c.close()
    assert n >= 10  # weights, moments, step, images, error word, average, Shampoo state
    assert abs(_free_bytes() - before) <= 8 << 20


def test_allocation_failure_in_training_and_batches():
    pool, tgt = synth.make_training_pool(8192, seed=5)
    P, T = torch.from_numpy(pool).to(DEV), torch.from_numpy(tgt).to(DEV)
    c = nrc.Cache(dtype="fp16", seed=6)
    before = _free_bytes()
    nrc.debug_fail_device_allocs(0, 1)  # the step's weight-gradient partials
    try:
        with pytest.raises(nrc.NrcError) as ei:
            c.train_step(P, T, 4096, synth.frame_seed(6, 0), 0)
    finally:
        nrc.debug_fail_device_allocs(0, 0)
    assert ei.value.status == nrc.NRC_ERR_OOM
    c.check_error()
    w0 = c.get_state()[0]
    c.train_step(P, T, 4096, synth.frame_seed(6, 0), 0)  # works once memory is there
    assert (c.get_state()[0] != w0).any()
    d = nrc.Cache(dtype="fp16", seed=7)
    n, b = _fail_each(lambda: nrc.Batch([c, d]))
    assert n >= 6
    b.close()
    d.close()
    c.close()
    assert abs(_free_bytes() - before) <= 8 << 20


def test_allocation_failure_in_server_viewport():
    srv = nrc.Server(nrc.default_config(dtype="fp16"))
    n, vp = _fail_each(lambda: srv.open_viewport(10_000, 4 * 16384, seed=1))
    assert n >= 1
    assert srv.info().viewports == 1
    srv.close_viewport(vp)
    assert srv.info().viewports == 0 and srv.info().memory_used == 0
    srv.close()


def test_allocation_failure_in_host_frames_is_resumable():
    # nrc_frame_host allocates its staging buffer, then (pipelined path) its
    # weight-image snapshot: fail each, then run the frame and compare it with
    # a frame from device buffers
    n_q = 70_000
    qn = synth.make_records(n_q, seed=8)
    pool, tgt = synth.make_training_pool(4096, seed=9)
    fs = synth.frame_seed(8, 0)
    a = nrc.Cache(dtype="fp16", seed=10)
    b = nrc.Cache(dtype="fp16", seed=10)
    qh, ph, th = (torch.from_numpy(x).pin_memory() for x in (qn, pool, tgt))
    rgb_h = torch.empty((n_q, 3)).pin_memory()
    for after in (0, 1):
        nrc.debug_fail_device_allocs(after, 1)
        try:
            with pytest.raises(nrc.NrcError) as ei:
                a.frame_host(qh, rgb_h, ph, th, 1024, 2, fs)
        finally:
            nrc.debug_fail_device_allocs(0, 0)
        assert ei.value.status == nrc.NRC_ERR_OOM
        # the frame's training had not started: the weights are untouched
        assert (a.get_state()[0] == b.get_state()[0]).all()
    a.frame_host(qh, rgb_h, ph, th, 1024, 2, fs)
    rgb_d = torch.empty((n_q, 3), device=DEV)
    b.frame(qh.to(DEV), rgb_d, ph.to(DEV), th.to(DEV), 1024, 2, fs)
    torch.cuda.synchronize()
    assert torch.equal(rgb_h, rgb_d.cpu())
    a.check_error()
