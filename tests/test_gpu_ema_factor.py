"""GPU parity of the weight average (Sec. 3.3, Eq. 2 as read) and of reflectance
factorisation (Sec. 5) against the FP64 oracle.

* the average kept by the Adam kernel equals the oracle's Eq. 2 recursion over
  the weights the GPU produced (FP32 arithmetic on both sides of one formula:
  1e-5 relative, floored at the rms);
* queries read the average, not the trained weights;
* on a fixed scene with noisy targets the average makes consecutive frames'
  outputs vary far less (synthetic analogue of the paper's temporal-stability
  figure, measured as SMAPE over consecutive frames);
* factorised queries and training steps match the oracle (fused FP32, plain
  FP32 and FP16 tensor-core paths) within the path's tolerance.
"""
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
DIMS = synth.layer_dims()
TOL = {"fp32": 1e-5, "fp16": 2e-2}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.mark.parametrize("dtype", ["fp32", "fp16"])
def test_average_follows_eq2_over_the_gpu_weights(dtype):
    c = nrc.Cache(dtype=dtype, ema=1, ema_alpha=0.99, seed=31)
    w0 = c.get_state()[0]
    assert np.array_equal(c.get_ema(), w0)  # before training the average is the weights
    pool, tgt = synth.make_training_pool(4 * 4096, seed=32)
    P, T = dev(pool), dev(tgt)
    e = w0.astype(np.float64)
    for f in range(3):
        for s in range(4):
            c.train_step(P, T, 4096, synth.frame_seed(33, f), s)
            w, _, _, t = c.get_state()
            e = O.ema(e, w, t, 0.99)
    got = c.get_ema()
    print("ema", dtype, stats(got, e))
    assert rel_err(got, e).max() <= 1e-5
    c.check_error()


@pytest.mark.parametrize("dtype", ["fp32", "fp16"])
def test_queries_read_the_average(dtype):
    c = nrc.Cache(dtype=dtype, ema=1, seed=41)
    pool, tgt = synth.make_training_pool(4 * 4096, seed=42)
    P, T = dev(pool), dev(tgt)
    for f in range(4):
        for s in range(4):
            c.train_step(P, T, 4096, synth.frame_seed(43, f), s)
    rec = synth.make_records(3000, seed=44)
    got = c.infer(dev(rec)).cpu().numpy()
    ema, w = c.get_ema(), c.get_state()[0]
    ref_ema, ref_w = O.infer(ema, DIMS, rec), O.infer(w, DIMS, rec)
    e_ema, e_w = rel_err(got, ref_ema).max(), rel_err(got, ref_w).max()
    print("query", dtype, "vs average", e_ema, "vs weights", e_w)
    assert e_ema <= TOL[dtype]
    assert e_w > 5 * e_ema


def _smape(a, b):
    return float(np.mean(2.0 * np.abs(a - b) / (np.abs(a) + np.abs(b) + 1e-6)))


def test_average_damps_frame_to_frame_variation():
    pool, clean = synth.make_training_pool(4 * 4096, seed=51)
    rng = np.random.default_rng(52)
    q = dev(synth.make_records(8192, seed=53))
    P = dev(pool)
    out = {}
    for use in (0, 1):
        c = nrc.Cache(dtype="fp16", ema=use, seed=54)
        rng = np.random.default_rng(52)
        frames = []
        for f in range(60):
            noisy = (clean * np.exp(0.5 * rng.normal(size=clean.shape))).astype(np.float32)
            c.frame(q[:0], q[:0], P, dev(noisy), 4096, 4, synth.frame_seed(55, f))
            frames.append(c.infer(q).cpu().numpy().astype(np.float64))
        c.check_error()
        out[use] = np.mean([_smape(frames[i], frames[i + 1]) for i in range(20, 59)])
    print("SMAPE consecutive frames: raw", out[0], "average", out[1])
    assert out[1] < 0.5 * out[0]


@pytest.mark.parametrize("dtype,path", [("fp32", nrc.PATH_FUSED), ("fp32", nrc.PATH_PLAIN), ("fp16", nrc.PATH_FUSED)])
def test_factorised_query_and_training_step(dtype, path):
    w0 = synth.xavier_weights(DIMS, seed=61)
    c = nrc.Cache(dtype=dtype, path=path, refl_factor=1, seed=61)
    c.set_state(w0)
    rec = synth.make_records(2000, seed=62)
    got = c.infer(dev(rec)).cpu().numpy()
    ref = O.infer(w0, DIMS, rec, refl_factor=True)
    assert rel_err(got, ref).max() <= TOL[dtype], stats(got, ref)
    assert rel_err(got, O.infer(w0, DIMS, rec)).max() > 10 * TOL[dtype]  # the factor is applied
    pool, tgt = synth.make_training_pool(8192, seed=63)
    loss = torch.zeros(1, device=DEV)
    c.train_step(dev(pool), dev(tgt), 4096, synth.frame_seed(64, 0), 1, loss_out=loss)
    st = O.TrainState(w0, DIMS)
    ref_loss, ref_g = st.step(pool, tgt, 4096, synth.frame_seed(64, 0), 1, refl_factor=True, want_grad=True)
    g = c.get_state()[1].astype(np.float64) / (1.0 - 0.9)
    print("factor", dtype, path, "loss", loss.item(), ref_loss, "grad", stats(g, ref_g))
    assert abs(loss.item() - ref_loss) <= TOL[dtype] * abs(ref_loss)
    bound = 1e-4 if dtype == "fp32" else 2e-2
    assert np.linalg.norm(g - ref_g) <= bound * np.linalg.norm(ref_g)
    c.check_error()


def test_batched_caches_with_average_and_factor_equal_single_caches():
    caches, recs = [], []
    for k in range(3):
        c = nrc.Cache(dtype="fp16", ema=1, refl_factor=1, seed=70 + k)
        pool, tgt = synth.make_training_pool(8192, seed=80 + k)
        for s in range(2):
            c.train_step(dev(pool), dev(tgt), 4096, synth.frame_seed(90 + k, 0), s)
        caches.append(c)
        recs.append(dev(synth.make_records(1000 + 777 * k, seed=100 + k)))
    single = [c.infer(r) for c, r in zip(caches, recs)]
    out = [torch.empty_like(s) for s in single]
    nrc.Batch(caches).infer(recs, out)
    torch.cuda.synchronize()
    for a, b in zip(out, single):
        assert torch.equal(a, b)
    with pytest.raises(nrc.NrcError):
        nrc.Batch([caches[0], nrc.Cache(dtype="fp16", seed=5)])  # mixed configurations


def test_allocation_free_step_rejects_the_average():
    cfg = nrc.default_config(dtype="fp16", ema=1)
    n = synth.n_params(DIMS)
    w = dev(np.zeros(n, np.float32))
    with pytest.raises(nrc.NrcError) as ei:
        nrc.train_step_noalloc(cfg, w, w.clone(), w.clone(), torch.zeros(1, dtype=torch.int64, device=DEV),
                               dev(np.zeros((256, 16), np.float32)), dev(np.zeros((256, 3), np.float32)), 128, 1, 0)
    assert ei.value.status == nrc.NRC_ERR_UNSUPPORTED
