"""Serving runtime on the GPU: continuous batching of several viewports' frames.

* a viewport's frame outputs, losses and final weights are bit-identical when
  it is served alone and when its frames share launches with other
  viewports' frames (every viewport trains with a CTA partition fixed by its
  own batch size);
* the first frame's outputs and first training loss agree with the FP64
  oracle within the 16-bit path's tolerance;
* viewports are admitted by memory: refused over the budget, admitted again
  once another closes; a slot still in flight refuses a new frame;
* a short Poisson-arrival run completes every frame with sane timings.
"""
import time

import numpy as np
import pytest

from paper_2106_12372_gb300 import synth
from parity import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2106_12372_gb300 import build, nrc  # noqa: E402

DEV = torch.device("cuda:0")
DIMS = synth.layer_dims()
STEPS, TBATCH = 2, 2048
FRAMES = 5
X_N, X_SEED = 5000, 11
OTHERS = [(1_000_000, 12), (3000, 13), (777, 14)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _server(**kw):
    kw.setdefault("train_steps", STEPS)
    kw.setdefault("train_batch", TBATCH)
    kw.setdefault("train_tiles", 4)
    return nrc.Server(nrc.default_config(dtype="fp16"), **kw)


def _fill_pool(srv, vid, seed):
    pool, tgt, _ = srv.pool(vid)
    p, t = synth.make_training_pool(pool.shape[0], seed=seed)
    pool.copy_(torch.from_numpy(p))
    tgt.copy_(torch.from_numpy(t))
    torch.cuda.synchronize()
    return p, t


X_RECS = [synth.make_records(X_N, seed=300 + f) for f in range(FRAMES)]


def _write(srv, vid, slot, rec):
    r, _, _ = srv.buffers(vid, slot)
    r[: rec.shape[0]].copy_(torch.from_numpy(rec) if isinstance(rec, np.ndarray) else rec)
    torch.cuda.synchronize()


def _run_x(srv, x, others):
    """Serves X's frames in order; other viewports' frames are submitted around them."""
    outs, losses, batch_sizes = {}, {}, []
    other_recs = {}
    for vid, n in others:
        rec = torch.from_numpy(synth.make_records(n, seed=400 + vid)).to(DEV)
        other_recs[vid] = (rec, n)
        for s in range(2):
            _write(srv, vid, s, rec)
    pending = {}

    def collect(block):
        got = srv.poll(timeout_ms=2000 if block else 0)
        if block and not got:
            raise AssertionError("no frame completed within 2 s")
        for d in got:
            assert not d.failed
            if d.viewport == x:
                _, rgb, ls = srv.buffers(x, d.slot)
                outs[d.tag] = rgb[:X_N].clone()
                losses[d.tag] = ls.clone()
                batch_sizes.append(d.batch_frames)
                torch.cuda.synchronize()
            pending.pop((d.viewport, d.slot), None)

    for f in range(FRAMES):
        slot = f % 2
        order = [vid for vid, _ in others] + [x]  # X last: it joins frames already pending
        for vid in order:  # the slot's previous frames finish first (the server is not held)
            while (vid, slot) in pending:
                collect(True)
        if others:
            srv.pause(True)  # the round's frames are released together: X shares their batch
        for vid in order:
            if vid == x:
                _write(srv, x, slot, X_RECS[f])
                ok = srv.submit(x, slot, X_N, synth.frame_seed(X_SEED, f), tag=f)
            else:
                ok = srv.submit(vid, slot, other_recs[vid][1], synth.frame_seed(vid, f), tag=f)
            assert ok
            pending[(vid, slot)] = True
        srv.pause(False)
    srv.drain()
    while len(outs) < FRAMES or pending:
        collect(True)
    w = srv.cache(x).get_state()
    return outs, losses, w, batch_sizes


def test_alone_equals_mixed():
    alone = _server()
    xa = alone.open_viewport(X_N, STEPS * TBATCH, seed=X_SEED)
    pool_np, tgt_np = _fill_pool(alone, xa, seed=X_SEED)
    out_a, loss_a, w_a, _ = _run_x(alone, xa, [])
    alone.close()

    mixed = _server()
    others = []
    for n, seed in OTHERS:
        vid = mixed.open_viewport(n, STEPS * TBATCH, seed=seed)
        _fill_pool(mixed, vid, seed=seed)
        others.append((vid, n))
    xm = mixed.open_viewport(X_N, STEPS * TBATCH, seed=X_SEED)
    _fill_pool(mixed, xm, seed=X_SEED)
    out_m, loss_m, w_m, bsz = _run_x(mixed, xm, others)
    info = mixed.info()
    mixed.close()

    assert max(bsz) > 1, "X never shared a batch with another viewport"
    assert info.frames_done == FRAMES * (len(OTHERS) + 1)
    for f in range(FRAMES):
        assert torch.equal(out_a[f], out_m[f]), f
        assert torch.equal(loss_a[f], loss_m[f]), f
    for a, b in zip(w_a[:3], w_m[:3]):
        assert np.array_equal(a, b)
    assert w_a[3] == w_m[3] == FRAMES * STEPS

    # frame 0 against the oracle: the query uses the initial Xavier weights,
    # and the first training step's loss is the oracle's on the same batch
    w0 = synth.xavier_weights(DIMS, seed=X_SEED)
    ref = O.infer(w0, DIMS, X_RECS[0])
    assert rel_err(out_a[0].cpu().numpy(), ref).max() <= 2e-2
    st = O.TrainState(w0, DIMS)
    ref_loss, _ = st.step(pool_np, tgt_np, TBATCH, synth.frame_seed(X_SEED, 0), 0, want_grad=True)
    assert abs(loss_a[0][0].item() - ref_loss) <= 2e-2 * abs(ref_loss)


def test_admission_by_memory():
    mq, n_pool = 200_000, STEPS * TBATCH
    per_vp = 2 * (mq * 64 + mq * 12) + n_pool * 76
    srv = _server(memory_budget=int(per_vp * 1.5))
    a = srv.open_viewport(mq, n_pool, seed=1)
    with pytest.raises(nrc.NrcError) as ei:
        srv.open_viewport(mq, n_pool, seed=2)
    assert ei.value.status == nrc.NRC_ERR_BUSY
    assert srv.info().viewports == 1
    used = srv.info().memory_used
    assert per_vp <= used <= srv.cfg.memory_budget
    # a slot in flight refuses a second frame
    _fill_pool(srv, a, seed=1)
    _write(srv, a, 0, synth.make_records(1000, seed=5))
    assert srv.submit(a, 0, 1000, 7)
    second = srv.submit(a, 0, 1000, 8)
    srv.drain()
    srv.poll()
    if second:  # the first frame may already have finished; then the slot was free again
        srv.drain()
    srv.close_viewport(a)
    assert srv.info().memory_used == 0
    b = srv.open_viewport(mq, n_pool, seed=2)
    assert srv.info().viewports == 1 and b >= 0
    srv.close()


def test_poisson_run_completes():
    srv = _server(train_steps=4, train_batch=4096)
    rng = np.random.default_rng(5)
    vps = []
    for k, n in enumerate([65536, 20000, 131072]):
        vid = srv.open_viewport(n, 4 * 4096, seed=50 + k)
        _fill_pool(srv, vid, seed=50 + k)
        rec = synth.make_records(n, seed=60 + k)
        for s in range(2):
            _write(srv, vid, s, rec)
        vps.append((vid, n, rng.uniform(30, 120)))
    arrivals = []
    for vid, n, rate in vps:
        t = rng.exponential(1 / rate)
        while t < 0.3:
            arrivals.append((t, vid, n))
            t += rng.exponential(1 / rate)
    arrivals.sort()
    t0 = nrc.now_ns()
    nxt = {vid: 0 for vid, _, _ in vps}
    busy = {}
    done = []
    for t, vid, n in arrivals:
        while nrc.now_ns() < t0 + int(t * 1e9):
            done += srv.poll(timeout_ms=0)
            time.sleep(0.0002)
        slot = nxt[vid] % 2
        deadline = time.monotonic() + 10.0
        while not srv.submit(vid, slot, n, synth.frame_seed(vid, nxt[vid]), arrival_ns=t0 + int(t * 1e9)):
            assert time.monotonic() < deadline, "slot never freed"
            done += srv.poll(timeout_ms=5)
        nxt[vid] += 1
        busy[vid] = True
    srv.drain()
    done += srv.poll(max_out=4096)
    srv.close()
    assert len(done) == len(arrivals)
    lat = np.array([(d.done_ns - d.arrival_ns) / 1e6 for d in done])
    assert np.all(lat > 0) and np.all(lat < 1000)
    assert all(d.launch_ns >= d.submit_ns and d.done_ns >= d.launch_ns for d in done)
    print("poisson frames", len(done), "p50 ms", np.percentile(lat, 50), "p99 ms", np.percentile(lat, 99))


def test_pause_holds_frames_until_released():
    srv = _server()
    vids = [srv.open_viewport(5000, STEPS * TBATCH, seed=s) for s in (31, 32, 33)]
    for k, v in enumerate(vids):
        _fill_pool(srv, v, seed=31 + k)
        _write(srv, v, 0, synth.make_records(5000, seed=40 + k))
    srv.pause(True)
    for v in vids:
        assert srv.submit(v, 0, 5000, synth.frame_seed(v, 0), tag=v)
    time.sleep(0.05)
    assert srv.poll(timeout_ms=20) == []  # held
    srv.pause(False)
    done = []
    while len(done) < 3:
        got = srv.poll(timeout_ms=2000)
        assert got, "released frames did not complete"
        done += got
    assert all(d.batch_frames == 3 for d in done)  # one batch
    # drain releases a held server
    for v in vids:
        _write(srv, v, 1, synth.make_records(5000, seed=50))
    srv.pause(True)
    for v in vids:
        assert srv.submit(v, 1, 5000, synth.frame_seed(v, 1), tag=10 + v)
    srv.drain()
    assert len(srv.poll(timeout_ms=0)) == 3
    srv.close()

