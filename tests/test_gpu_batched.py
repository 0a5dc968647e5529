"""Batched caches (several independent caches served together) on the GPU.

* one persistent query launch over caches with uneven query counts gives, row
  for row, exactly the single-cache result (same arithmetic per row);
* one batched training step matches the FP64 oracle per cache, within the
  16-bit path's tolerance;
* the autotuner picks a candidate work-unit size and the results do not
  depend on it; the batched query replays from a captured CUDA graph.
"""
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
DIMS = synth.layer_dims()
NS = [1, 127, 129, 1000, 0, 40_000, 262_144, 5_003]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def setup():
    build.build()
    caches, recs, ws = [], [], []
    for k, n in enumerate(NS):
        c = nrc.Cache(dtype="fp16", seed=500 + k)
        w = synth.xavier_weights(DIMS, seed=500 + k)
        c.set_state(w)
        caches.append(c)
        ws.append(w)
        recs.append(dev(synth.make_records(max(n, 0), seed=600 + k)))
    return caches, recs, ws


def _single(caches, recs):
    return [c.infer(r) if r.shape[0] else torch.empty((0, 3), device=DEV) for c, r in zip(caches, recs)]


@pytest.mark.parametrize("unit", [0, 1, 7, 20, 160])
def test_batch_infer_equals_single_cache(setup, unit):
    caches, recs, _ = setup
    ref = _single(caches, recs)
    b = nrc.Batch(caches)
    b.set_unit_tiles(unit)
    out = [torch.full((r.shape[0], 3), float("nan"), device=DEV) for r in recs]
    b.infer(recs, out)
    torch.cuda.synchronize()
    for k in range(len(NS)):
        assert torch.equal(out[k], ref[k]), (unit, k)
    for c in caches:
        c.check_error()


def test_batch_infer_matches_oracle(setup):
    caches, recs, ws = setup
    b = nrc.Batch(caches)
    out = [torch.empty((r.shape[0], 3), device=DEV) for r in recs]
    b.infer(recs, out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for k, n in enumerate(NS):
        if n == 0:
            continue
        idx = rng.choice(n, min(n, 500), replace=False)
        ref = O.infer(ws[k], DIMS, recs[k].cpu().numpy()[idx])
        assert rel_err(out[k].cpu().numpy()[idx], ref).max() <= 2e-2, k


def test_batch_autotune_and_graph_replay(setup):
    caches, recs, _ = setup
    ref = _single(caches, recs)
    b = nrc.Batch(caches)
    out = [torch.empty((r.shape[0], 3), device=DEV) for r in recs]
    chosen = b.autotune(recs, out)
    assert chosen in (0, 5, 10, 20, 40, 80, 160)
    b.infer(recs, out)  # uploads the descriptors for this unit size before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for o in out:
            o.fill_(float("nan"))
        with torch.cuda.graph(g, stream=s):
            b.infer(recs, out, stream=s)
    for o in out:
        o.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for k in range(len(NS)):
        assert torch.equal(out[k], ref[k]), k


def test_batch_train_step_matches_oracle():
    build.build()
    batches = [16384, 4096, 1000, 65536 // 4]
    caches, states, pools, tgts, fss = [], [], [], [], []
    for k, bs in enumerate(batches):
        w = synth.xavier_weights(DIMS, seed=700 + k)
        c = nrc.Cache(dtype="fp16", seed=700 + k)
        c.set_state(w)
        caches.append(c)
        states.append(O.TrainState(w, DIMS))
        p, t = synth.make_training_pool(bs * 4, seed=800 + k)
        pools.append(p)
        tgts.append(t)
        fss.append(synth.frame_seed(900 + k, 0))
    b = nrc.Batch(caches)
    losses = [torch.zeros(1, device=DEV) for _ in caches]
    b.train_step([dev(p) for p in pools], [dev(t) for t in tgts], batches, fss, 2, losses)
    torch.cuda.synchronize()
    for k, c in enumerate(caches):
        ref_loss, ref_g = states[k].step(pools[k], tgts[k], batches[k], fss[k], 2, want_grad=True)
        w, m, v, t = c.get_state()
        g = m.astype(np.float64) / (1.0 - 0.9)
        print("batched train", k, batches[k], stats(g, ref_g))
        assert t == 1
        assert abs(losses[k].item() - ref_loss) <= 2e-2 * abs(ref_loss)
        assert np.linalg.norm(g - ref_g) <= 2e-2 * np.linalg.norm(ref_g)
        # and per element, the format tolerance of the batch the cache trained on
        rec, tg, _ = O.gather(pools[k], tgts[k], batches[k], fss[k], 2)
        emul = EB.emulate_16bit(synth.xavier_weights(DIMS, seed=700 + k), DIMS, O.encode(rec), tg, "fp16")[1]
        EB.format_check(g, ref_g, emul, DIMS, label=f"batched train {k}")
        c.check_error()


def test_batch_rejects_mixed_configurations():
    build.build()
    a = nrc.Cache(dtype="fp16")
    b16 = nrc.Cache(dtype="bf16")
    with pytest.raises(nrc.NrcError):
        nrc.Batch([a, b16])
    f32 = nrc.Cache(dtype="fp32")
    with pytest.raises(nrc.NrcError):
        nrc.Batch([f32])



def _i64(seeds):
    return torch.tensor([x - (1 << 64) if x >= 1 << 63 else x for x in seeds], dtype=torch.int64)


def test_batch_train_step_dev_equals_host_seeds_and_replays_in_a_graph():
    """Frame seeds in device memory: the same bits as host seeds, eagerly and
    from one captured graph (query launch + gradient launch + Adam launch)
    replayed with new seeds written before each replay -- one training step
    per frame, as the batched-caches frame runs it."""
    bl = [4096, 129, 20_000]
    pools, tgts = [], []
    for k, n in enumerate(bl):
        p, t = synth.make_training_pool(2 * n, seed=900 + k)
        pools.append(dev(p))
        tgts.append(dev(t))
    recs = [dev(synth.make_records(n, seed=950 + k)) for k, n in enumerate((1000, 129, 5000))]
    seeds = [[synth.frame_seed(970 + k, f) for k in range(3)] for f in range(3)]

    ref_c = [nrc.Cache(dtype="fp16", seed=980 + k) for k in range(3)]
    ref_b = nrc.Batch(ref_c)
    ref_out = []
    for f in range(3):
        out = [torch.empty((r.shape[0], 3), device=DEV) for r in recs]
        ref_b.infer(recs, out)
        ref_b.train_step(pools, tgts, bl, seeds[f], 0)
        ref_out.append(out)
    torch.cuda.synchronize()

    got_c = [nrc.Cache(dtype="fp16", seed=980 + k) for k in range(3)]
    got_b = nrc.Batch(got_c)
    sd = torch.zeros(3, dtype=torch.int64, device=DEV)
    out = [torch.empty((r.shape[0], 3), device=DEV) for r in recs]
    got_out = []
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sd.copy_(_i64(seeds[0]))
        got_b.infer(recs, out, stream=s)
        got_b.train_step_dev(pools, tgts, bl, sd, 0, stream=s)  # uploads the descriptors
        got_out.append([o.clone() for o in out])
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            got_b.infer(recs, out, stream=s)
            got_b.train_step_dev(pools, tgts, bl, sd, 0, stream=s)
        for f in (1, 2):
            sd.copy_(_i64(seeds[f]))
            g.replay()
            got_out.append([o.clone() for o in out])
        s.synchronize()
    for f in range(3):
        for k in range(3):
            assert torch.equal(got_out[f][k], ref_out[f][k]), (f, k)
    for a, b in zip(ref_c, got_c):
        a.check_error()
        b.check_error()
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    for c in ref_c + got_c:
        c.close()
    ref_b.close()
    got_b.close()


def test_batch_train_more_caches_than_sms():
    """160 one-tile caches: their training CTAs do not fit one per SM, so the
    training launches run whole caches in turn; each cache's result equals
    its training alone, bit for bit (its partition and sums do not depend on
    the others)."""
    nc = 160
    ps, ts = [], []
    for k in range(nc):
        p, t = synth.make_training_pool(256, seed=1200 + k)
        ps.append(dev(p))
        ts.append(dev(t))
    fss = [synth.frame_seed(1300 + k, 0) for k in range(nc)]
    mixed = [nrc.Cache(dtype="fp16", seed=1400 + k) for k in range(nc)]
    nrc.Batch(mixed).train_step(ps, ts, [128] * nc, fss, 1)
    torch.cuda.synchronize()
    for k in range(0, nc, 23):
        alone = nrc.Cache(dtype="fp16", seed=1400 + k)
        nrc.Batch([alone]).train_step([ps[k]], [ts[k]], [128], [fss[k]], 1)
        for x, y in zip(mixed[k].get_state(), alone.get_state()):
            assert np.array_equal(np.asarray(x), np.asarray(y)), k
        alone.close()
    for c in mixed:
        c.check_error()
        c.close()
