"""GPU parity of the training-record pipeline (Sec. 3.3-3.5; termination
heuristic Eqs. 3-4) against the oracle on seeded synthetic paths.

The oracle takes the termination decisions in FP64 from the definition; the
GPU's (FP32) must equal them except for decisions within the FP32 band of the
threshold (oracle.paths_check_decisions), of which at most MAX_DIFFER may go
the other way.  Given the decisions, the training tiles and every record are
bit-exact; emitted sums, throughputs, targets and the composite agree to 1e-5
(FP32 against FP64, floored at the rms).
"""
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
W, H, K = 97, 61, 10
MAX_DIFFER = 3


def _ends(v, rq):
    """The vertex index each pixel's query record was taken from (bitwise match)."""
    rec = rq.cpu().numpy()[:, :14].view(np.uint32)
    eq = np.all(v[:, :, :14].view(np.uint32) == rec[:, None, :], axis=2)
    assert np.all(eq.sum(axis=1) >= 1)
    return np.argmax(eq, axis=1)


def _checked(v, rq, tiles, c, tile, ox, oy, phase):
    n = _ends(v, rq)
    t = tiles.cpu().numpy()
    ok, differ = O.paths_check_decisions(v, W, H, synth.PATH_CAMERA, c, tile, ox, oy, phase, 0.8, n, t)
    print("termination decisions taken the other way (within the FP32 band):", differ)
    assert ok and differ <= MAX_DIFFER, differ
    return n, [tuple(r) for r in t.tolist()]


@pytest.fixture(scope="module")
def scene():
    build.build()
    v = synth.make_paths(W, H, K, seed=21)
    return v, torch.from_numpy(v).to(DEV)


def _params(c=0.01, tile=8, ox=3, oy=5, phase=7, q=0.8):
    return nrc.PathParams(c, tile, ox, oy, phase, q)


def _record(vtx_row):
    r = np.zeros(16, np.float32)
    r[:14] = vtx_row[:14]
    return r


@pytest.mark.parametrize("c,tile,ox,oy,phase", [(0.01, 8, 3, 5, 7), (0.1, 5, 0, 4, -1), (0.001, 16, 15, 15, 0)])
def test_termination_and_tiles_match_oracle(scene, c, tile, ox, oy, phase):
    v, V = scene
    rq, em, tp, tiles, tq = nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, _params(c, tile, ox, oy, phase))
    n, ref_tiles = _checked(v, rq, tiles, c, tile, ox, oy, phase)
    E, T = O.paths_radiance(v, n)
    ref_rq = np.stack([_record(v[p, n[p]]) for p in range(W * H)])
    assert np.array_equal(rq.cpu().numpy().view(np.uint32), ref_rq.view(np.uint32))
    tqh = tq.cpu().numpy()
    for t, (p, nn, m, unb) in enumerate(ref_tiles):
        if p >= 0:
            assert np.array_equal(tqh[t].view(np.uint32), _record(v[p, m]).view(np.uint32))
    assert rel_err(em.cpu().numpy(), E).max() <= 1e-5
    assert rel_err(tp.cpu().numpy(), T).max() <= 1e-5
    assert (np.array(ref_tiles)[:, 0] >= 0).sum() > 10 and 0 < n.min() and n.max() <= K - 1


# tile 8: 104 tiles (one scan block); tile 1: every pixel trains, 5,917 tiles
# (three scan blocks of 2,048, the last one ragged)
@pytest.mark.parametrize("tile,ox,oy,phase,max_records", [(8, 3, 5, 7, 4096), (1, 0, 0, 5, 1 << 16)])
def test_records_and_targets_match_oracle(scene, tile, ox, oy, phase, max_records):
    v, V = scene
    prm = _params(tile=tile, ox=ox, oy=oy, phase=phase)
    rq, _, _, tiles, tq = nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, prm)
    _, ref_tiles = _checked(v, rq, tiles, 0.01, tile, ox, oy, phase)
    w0 = synth.xavier_weights(DIMS, seed=22)
    tail = O.infer(w0, DIMS, tq.cpu().numpy())  # the cache's values at the tails (FP64 oracle)
    ref_rec, ref_tg = O.paths_records(v, ref_tiles, tail, 0.8)
    pool, tg, count = nrc.paths_records(V, W, H, synth.PATH_CAMERA, prm, tiles,
                                        torch.from_numpy(tail.astype(np.float32)).to(DEV), max_records)
    N = len(ref_rec)
    assert count.item() == N and N > 50
    assert np.array_equal(pool[:N].cpu().numpy().view(np.uint32), ref_rec.view(np.uint32))
    assert rel_err(tg[:N].cpu().numpy(), ref_tg).max() <= 1e-5
    assert not pool[N:].any()
    # truncation: the first max_records are written, the count is the total
    pool2, tg2, count2 = nrc.paths_records(V, W, H, synth.PATH_CAMERA, prm, tiles,
                                           torch.from_numpy(tail.astype(np.float32)).to(DEV), N // 3)
    assert count2.item() == N
    assert torch.equal(pool2, pool[:N // 3]) and torch.equal(tg2, tg[:N // 3])


def test_composite_matches_oracle(scene):
    v, V = scene
    _, em, tp, _, _ = nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, _params())
    rgb = np.random.default_rng(23).uniform(0, 2, size=(W * H, 3)).astype(np.float32)
    img = nrc.paths_composite(em, tp, torch.from_numpy(rgb).to(DEV)).cpu().numpy()
    ref = O.paths_composite(em.cpu().numpy(), tp.cpu().numpy(), rgb)
    assert rel_err(img, ref).max() <= 1e-6


def test_frame_through_the_cache(scene):
    v, V = scene
    cache = nrc.Cache(dtype="fp16", seed=24)
    tile = 4
    for f in range(6):
        prm = _params(tile=tile, ox=f % tile, oy=(3 * f) % tile, phase=f % 16)
        rq, em, tp, tiles, tq = nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, prm)
        rgb = cache.infer(rq)
        tail = cache.infer(tq)
        pool, tg, count = nrc.paths_records(V, W, H, synth.PATH_CAMERA, prm, tiles, tail, 1 << 14)
        n = int(count.item())
        assert 0 < n <= 1 << 14
        batch = n // 4
        cache.frame(rq[:0], rgb[:0], pool[:n], tg[:n], batch, 4, synth.frame_seed(25, f))
        img = nrc.paths_composite(em, tp, rgb)
        assert torch.isfinite(img).all()
        tile = nrc.paths_adapt_tile(tile, n, 2048)
    cache.check_error()


def test_preallocated_outputs_match(scene):
    v, V = scene
    prm = _params(tile=6, ox=2, oy=1, phase=3)
    ref = nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, prm)
    nt = nrc.paths_tile_count(W, H, 6)
    out = (torch.empty((W * H, 16), device=DEV), torch.empty((W * H, 3), device=DEV),
           torch.empty((W * H, 3), device=DEV), torch.empty((nt, 4), dtype=torch.int32, device=DEV),
           torch.zeros((nt, 16), device=DEV))
    got = nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, prm, out=out)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    tail = torch.rand((nt, 3), device=DEV, generator=torch.Generator(device=DEV).manual_seed(5))
    pr, tr, cr = nrc.paths_records(V, W, H, synth.PATH_CAMERA, prm, ref[3], tail, 4096)
    bufs = (torch.full((4096, 16), 7.0, device=DEV), torch.full((4096, 3), 7.0, device=DEV),
            torch.empty(nrc.paths_offsets_count(nt), dtype=torch.int64, device=DEV),
            torch.zeros(1, dtype=torch.int64, device=DEV))
    pg, tg_, cg = nrc.paths_records(V, W, H, synth.PATH_CAMERA, prm, ref[3], tail, 4096, out=bufs)
    n = int(cr.item())
    assert int(cg.item()) == n and 0 < n <= 4096
    assert torch.equal(pg[:n], pr[:n]) and torch.equal(tg_[:n], tr[:n])
    img = torch.empty((W * H, 3), device=DEV)
    assert torch.equal(nrc.paths_composite(ref[1], ref[2], tail[:1].expand(W * H, 3).contiguous(), out=img),
                       nrc.paths_composite(ref[1], ref[2], tail[:1].expand(W * H, 3).contiguous()))
    with pytest.raises(ValueError):
        nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, prm, out=(out[0][:10],) + out[1:])


def test_tail_queries_in_the_render_buffer():
    # the tail queries written after the render queries in one buffer, answered
    # by one query launch, equal the separate buffers and launches
    v = synth.make_paths(W, H, K, seed=21)
    V = torch.from_numpy(v).to(DEV)
    prm = _params(tile=5, ox=1, oy=4, phase=2)
    rq, em, tp, tiles, tq = nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, prm)
    nt = nrc.paths_tile_count(W, H, 5)
    P = W * H
    q_all = torch.zeros((P + nt, 16), device=DEV)
    t2 = torch.empty((nt, 4), dtype=torch.int32, device=DEV)
    nrc.paths_terminate(V, W, H, synth.PATH_CAMERA, prm,
                        out=(q_all[:P], torch.empty_like(em), torch.empty_like(tp), t2, q_all[P:]))
    assert torch.equal(q_all[:P], rq) and torch.equal(q_all[P:], tq) and torch.equal(t2, tiles)
    c = nrc.Cache(dtype="fp16", seed=27)
    both = c.infer(q_all)
    assert torch.equal(both[:P], c.infer(rq)) and torch.equal(both[P:], c.infer(tq))
    c.check_error()
