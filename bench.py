"""Benchmark of the neural radiance cache frame on GB300.

One step = one 1080p frame of the cache's hot path (Sec. 3.1-3.5): the cache
query for 1920 x 1080 = 2,073,600 path vertices, then 4 training steps of
16,384 records each drawn (shuffled, disjoint) from the frame's 65,536-record
pool, FP16 tensor-core products with FP32 accumulation and FP32 master weights
and Adam state.  Inputs are seeded synthetic records shaped like the paper's
workload (records U[0,1]^3 positions, directions and normals uniform on the
sphere, roughness and albedos U[0,1]; targets from an analytic HDR field).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead
(a deliberately slow correctness reference, bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUERIES = 1920 * 1080
BATCH = 16384
N_STEPS = 4
N_POOL = BATCH * N_STEPS
FLOP_QUERY = 2 * 20672          # forward pass, multiply-adds x 2
FLOP_QUERY_W128 = 2 * (64 * 128 + 6 * 128 * 128 + 128 * 3)  # width 128, 7 hidden layers
FLOP_RECORD = 41344 + 33152 + 41344  # forward + backward data + weight gradients
METRIC = "ms/frame and Mqueries/s (infer+train) fused vs plain FP32 path; % tensor peak; p99 frame ms"
WORKLOAD = ("1080p frame: 2,073,600 cache queries + 4 train steps x 16,384 records from a 65,536-record pool; "
            "width-64 5-hidden-layer MLP, 64-dim encoding (cheap primitives, pad 1)")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), d.get("hbm_gbs", 6800.0), "measured"
    return 1900.0, 1700.0, 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 20 ms while running (the
    benchmark runs 0.3 s of untimed frames inside it before the timed ones, so
    the record is taken under the frame's load however short the timed region)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = [ln.split(",") for ln in self.out.strip().splitlines() if ln.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def frame_traffic():
    """DRAM bytes per k_frame_tc launch from the committed ncu summary, or None
    once the kernel's sources differ from the ones that were profiled."""
    import hashlib
    import re

    prof = os.path.join(ROOT, "profiles", "k_frame_tc_1080p_fp16.md")
    if not os.path.exists(prof):
        return None
    text = open(prof).read()
    mt = re.search(r"^traffic_bytes_per_launch: (\d+)", text, re.M)
    mh = re.search(r"^source_sha256_16: ([0-9a-f]{16})", text, re.M)
    if not (mt and mh):
        return None
    csrc = os.path.join(ROOT, "paper_2106_12372_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("k_frame.cu", "tc_common.cuh", "tc_ptx.cuh", "nrc_internal.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return int(mt.group(1)) if h.hexdigest()[:16] == mh.group(1) else None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_throughput(local_ms: float, units_per_rank: int, steps: int, ws: int, device=None):
    """The timed region's length as the MAX over ranks, and whole-job throughput
    in millions of units per second: the units all ranks processed over it."""
    import torch

    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    return total_ms, units_per_rank * steps * ws / (total_ms / 1e3) / 1e6


def build_once(ws: int, rank: int, build_fn) -> bool:
    """Rank 0 runs build_fn while the other ranks wait on the host (a gloo
    group, so no rank sits in a device collective meanwhile); every rank then
    learns whether it succeeded.  Returns that outcome (True on one rank when
    build_fn returns)."""
    if ws == 1:
        build_fn()
        return True
    import torch
    import torch.distributed as dist

    group = dist.new_group(backend="gloo")
    ok = torch.zeros(1, dtype=torch.int32)
    if rank == 0:
        try:
            build_fn()
            ok[0] = 1
        except Exception as exc:  # reported by every rank through the flag
            sys.stderr.write(f"rank 0 build failed: {exc}\n")
    dist.broadcast(ok, src=0, group=group)
    return bool(ok.item())


_ORACLE_COST = {}


def _oracle_costs(seed: int):
    """Seconds per query and per training record of the FP64 oracle on this
    host, from one mid-sized call each (probed once; used to size samples)."""
    if not _ORACLE_COST:
        from oracle import oracle as O
        from paper_2106_12372_gb300 import synth

        dims = synth.layer_dims()
        w0 = synth.xavier_weights(dims, seed=seed)
        O.lib()
        rec = synth.make_records(32768, seed=seed + 1)
        pool, tgt = synth.make_training_pool(8192, seed=seed + 1)
        t0 = time.perf_counter()
        O.infer(w0, dims, rec)
        _ORACLE_COST["query"] = (time.perf_counter() - t0) / 32768
        st = O.TrainState(w0, dims)
        t0 = time.perf_counter()
        st.step(pool, tgt, 4096, synth.frame_seed(seed, 0), 0)
        _ORACLE_COST["record"] = (time.perf_counter() - t0) / 4096
    return _ORACLE_COST["query"], _ORACLE_COST["record"]


def cpu_oracle_frame(budget_s: float, seed: int = 2106):
    """Times the FP64 oracle on a bounded sample of the frame, about budget_s
    seconds of CPU work: whole frames (the frame's queries against the current
    weights, then its training steps) repeated while the budget lasts, or, for
    a budget below one frame, a share of the queries and smaller training
    batches in the frame's proportions, scaled to the frame (the oracle's cost
    per query falls with the batch it is given: 7.4 us at 2,048 queries, 2.8 us
    at a whole frame on 8 x86 cores, so small samples read low).  Returns
    (Mqueries/s, description, cores, ms per frame)."""
    from oracle import oracle as O
    from paper_2106_12372_gb300 import synth

    t_q, t_r = _oracle_costs(seed)
    full = N_QUERIES * t_q + N_STEPS * BATCH * t_r
    share = min(1.0, budget_s / full)
    nq = int(max(1024, share * N_QUERIES))
    nb = int(max(256, share * BATCH))
    dims = synth.layer_dims()
    key = ("inputs", nq)
    if key not in _ORACLE_COST:  # the seeded inputs, drawn once per sample size
        _ORACLE_COST[key] = (synth.make_records(nq, seed=seed + 2), synth.make_training_pool(N_POOL, seed=seed + 3),
                             synth.xavier_weights(dims, seed=seed))
    rec, (pool, tgt), w0 = _ORACLE_COST[key]
    st = O.TrainState(w0, dims)
    frames, t_inf, t_tr = 0, 0.0, 0.0
    t_start = time.perf_counter()
    while frames == 0 or (time.perf_counter() - t_start) + (t_inf + t_tr) / frames <= budget_s:
        t0 = time.perf_counter()
        O.infer(st.W, dims, rec)
        t1 = time.perf_counter()
        for k in range(N_STEPS):
            st.step(pool, tgt, nb, synth.frame_seed(seed, frames), k)
        t_inf += t1 - t0
        t_tr += time.perf_counter() - t1
        frames += 1
    frame_s = (t_inf / frames) * (N_QUERIES / nq) + (t_tr / frames) * (BATCH / nb)
    cores = int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))
    what = ("whole frames" if nq == N_QUERIES and nb == BATCH else
            f"{nq} queries + {N_STEPS} steps of {nb} records each, scaled to the frame")
    desc = (f"{frames} x ({what}; frame = {N_QUERIES} queries + {N_STEPS} steps of {BATCH}); "
            f"oracle wall {t_inf + t_tr:.1f} s")
    return N_QUERIES / frame_s / 1e6, desc, cores, frame_s * 1e3


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    values = []
    descs = []
    cores = 1
    # about args.ref_seconds (90 s) of oracle work in all, however many steps are asked for
    per = max(0.05, args.ref_seconds / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        v, d, cores, _ = cpu_oracle_frame(per)
        if i >= args.warmup:
            values.append(v)
            descs.append(d)
    v = statistics.median(values)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mqueries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": N_QUERIES / (v * 1e6) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "Mqueries/s", "cores": cores, "kind": "oracle", "sample": descs[-1]},
            "e2e": {"value": v, "unit": "Mqueries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(queries, dtype: str, frames: int, flush):
    """16 independent caches in one persistent query launch (replayed from a
    CUDA graph) and one batched training step per frame.  Per-frame query
    counts are log-uniform in [4,096, 2,097,152] and training batches
    log-uniform in [4,096, 65,536] (seed 2110); cache k has its own weights
    and target field (seed 2106 + 100 k).  Query records are views into the
    two 2,073,600-record sets of the frame benchmark."""
    import numpy as np
    import torch

    from paper_2106_12372_gb300 import nrc, synth

    dev = queries[0].device
    rng = np.random.default_rng(2106 + 4)
    nq = np.exp(rng.uniform(np.log(4096), np.log(2097152), 16)).round().astype(np.int64)
    bt = np.exp(rng.uniform(np.log(4096), np.log(65536), 16)).round().astype(np.int64)
    allq = torch.cat(queries)
    recs, rgbs, pools, tgts, caches = [], [], [], [], []
    for k in range(16):
        off = (k * 262144) % (allq.shape[0] - int(nq[k]))
        recs.append(allq[off: off + int(nq[k])])
        rgbs.append(torch.empty((int(nq[k]), 3), device=dev))
        p, t = synth.make_training_pool(int(bt[k]), seed=2106 + 100 * k)
        pools.append(torch.from_numpy(p).to(dev))
        tgts.append(torch.from_numpy(t).to(dev))
        caches.append(nrc.Cache(dtype=dtype, seed=2106 + 100 * k))
    losses = [torch.zeros(1, device=dev) for _ in range(16)]
    s = torch.cuda.Stream()
    b = nrc.Batch(caches)
    bl = [int(x) for x in bt]
    sd = torch.zeros(16, dtype=torch.int64, device=dev)  # this frame's seeds, read by the gradient kernel

    def seeds(f):
        v = [synth.frame_seed(2106 + 100 * k, f) for k in range(16)]
        return torch.tensor([x - (1 << 64) if x >= 1 << 63 else x for x in v], dtype=torch.int64)

    with torch.cuda.stream(s):
        unit = b.autotune(recs, rgbs, stream=s)
        b.infer(recs, rgbs, stream=s)
        sd.copy_(seeds(0))
        b.train_step_dev(pools, tgts, bl, sd, 0, losses, stream=s)  # uploads the step's descriptors
        s.synchronize()
        # the whole frame -- query launch, gradient launch, Adam launch -- in one graph; and the query
        # launch alone in another, to split the frame's time between queries and training
        gq = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gq, stream=s):
            b.infer(recs, rgbs, stream=s)
        gf = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gf, stream=s):
            b.infer(recs, rgbs, stream=s)
            b.train_step_dev(pools, tgts, bl, sd, 0, losses, stream=s)

        def frame(f, ev=None):
            sd.copy_(seeds(f))  # 128 bytes host -> device, outside the events
            if ev:
                ev[0].record(s)
            gf.replay()
            if ev:
                ev[1].record(s)

        for f in range(3):
            frame(1 + f)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(frames)]
        for f in range(frames):
            flush.zero_()
            frame(4 + f, evs[f])
        qev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(frames)]
        for f in range(frames):
            flush.zero_()
            qev[f][0].record(s)
            gq.replay()
            qev[f][1].record(s)
        # the same work as 16 separate caches, one query and one training call each
        sev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(5)]
        for f in range(5):
            flush.zero_()
            sev[f][0].record(s)
            for k in range(16):
                caches[k].infer(recs[k], rgbs[k], stream=s)
                caches[k].train_step(pools[k], tgts[k], bl[k], synth.frame_seed(2106 + 100 * k, 100 + f), 0,
                                     loss_out=losses[k], stream=s)
            sev[f][1].record(s)
        s.synchronize()
    for c in caches:
        c.check_error()
    ms = [e[0].elapsed_time(e[1]) for e in evs]
    inf = [e[0].elapsed_time(e[1]) for e in qev]
    seq = [e[0].elapsed_time(e[1]) for e in sev[1:]]
    q = int(nq.sum())
    qflop, tflop = FLOP_QUERY * q, FLOP_RECORD * int(bt.sum())
    med, qmed = statistics.median(ms), statistics.median(inf)
    b.close()
    for c in caches:
        c.close()
    return {
        "workload": "16 caches: queries log-uniform [4096, 2097152], one training step of log-uniform [4096, 65536] "
                    "records each; the whole frame (query, gradient and Adam launches) replayed from one CUDA "
                    "graph, this frame's seeds written to the device before each replay; L2 flushed between frames",
        "queries": q, "train_records": int(bt.sum()), "frames": frames,
        "ms_median": med, "ms_p99": float(np.percentile(ms, 99)), "infer_ms_median": qmed,
        "train_ms_median": med - qmed,
        "mqueries_per_s": q / (med / 1e3) / 1e6, "tflops": (qflop + tflop) / (med / 1e3) / 1e12,
        "query_tflops": qflop / (qmed / 1e3) / 1e12,
        "train_tflops": tflop / ((med - qmed) / 1e3) / 1e12 if med > qmed else None,
        "split_note": "query time from the query launch alone (its own graph); training = frame - query",
        "unit_tiles_autotuned": unit, "launches_per_frame": 3, "launches_in_graph": 3,
        "sequential_16_caches_ms_median": statistics.median(seq),
    }


def run_shampoo(pool, tgt, dtype: str, frames: int, flush):
    """The frame's 4 training steps with Shampoo (roots once per frame) against
    Adam on the same pool: milliseconds per frame of training."""
    import numpy as np
    import torch

    from paper_2106_12372_gb300 import nrc, synth

    out = {}
    st = torch.cuda.current_stream()
    for name, opt in (("adam", nrc.OPT_ADAM), ("shampoo", nrc.OPT_SHAMPOO)):
        c = nrc.Cache(dtype=dtype, optimizer=opt, seed=2106)
        for f in range(3):
            c.frame(pool[:0], pool[:0], pool, tgt, BATCH, N_STEPS, synth.frame_seed(2106, f))
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(frames)]
        for f in range(frames):
            flush.zero_()
            ev[f][0].record(st)
            c.frame(pool[:0], pool[:0], pool, tgt, BATCH, N_STEPS, synth.frame_seed(2106, 3 + f))
            ev[f][1].record(st)
        torch.cuda.synchronize()
        c.check_error()
        out[name + "_train_ms_per_frame"] = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        c.close()
    out["workload"] = "4 training steps x 16,384 records per frame; Shampoo roots recomputed once per frame"
    return out


def run_precision(queries, flush, frames: int = 30):
    """Query time of the 1080p frame per arithmetic type, and each type's
    per-output error on a 2,000-query sample against the FP32 query path
    (median and max, relative to the sample rms floor; the FP32 path itself is
    held within 1e-5 of the FP64 oracle by the parity tests)."""
    import numpy as np
    import torch

    from paper_2106_12372_gb300 import nrc, synth

    dims = synth.layer_dims()
    w0 = synth.xavier_weights(dims, seed=2106)
    sample = queries[0][:2000]
    out = {}
    ref = None
    st = torch.cuda.current_stream()
    rgb = torch.empty((queries[0].shape[0], 3), device=queries[0].device)
    for dt in ("fp32", "bf16", "fp16", "fp8"):
        c = nrc.Cache(dtype=dt, seed=2106)
        c.set_state(w0)
        got = c.infer(sample).cpu().numpy().astype(np.float64)
        if ref is None:
            ref = got
            tau = np.sqrt(np.mean(ref ** 2))
        err = np.abs(got - ref) / np.maximum(np.abs(ref), tau)
        for k in range(3):
            c.infer(queries[k % 2], rgb)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(frames if dt != "fp32" else 5)]
        for k, e in enumerate(ev):
            flush.zero_()
            e[0].record(st)
            c.infer(queries[k % 2], rgb)
            e[1].record(st)
        torch.cuda.synchronize()
        c.check_error()
        ms = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        out[dt] = {"infer_ms": ms, "tflops": FLOP_QUERY * N_QUERIES / (ms / 1e3) / 1e12}
        if dt != "fp32":
            out[dt].update(err_median=float(np.median(err)), err_max=float(err.max()))
        c.close()
    # the wide variant: width 128, 7 hidden layers, on the plain per-layer FP32 path
    c = nrc.Cache(dtype="fp32", path=nrc.PATH_PLAIN, width=128, hidden_layers=7, seed=2106)
    c.infer(queries[0], rgb)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3)]
    for k, e in enumerate(ev):
        flush.zero_()
        e[0].record(st)
        c.infer(queries[k % 2], rgb)
        e[1].record(st)
    torch.cuda.synchronize()
    c.check_error()
    ms = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
    out["fp32_width128_7hidden"] = {"infer_ms": ms, "tflops": FLOP_QUERY_W128 * N_QUERIES / (ms / 1e3) / 1e12}
    w128 = c.get_state()[0]
    ref128 = c.infer(sample).cpu().numpy().astype(np.float64)
    c.close()
    # ... and its FP16 / BF16 queries on the tensor cores (k_tc128), against the plain FP32 path
    burst = peaks()[0]
    tau128 = np.sqrt(np.mean(ref128 ** 2))
    for dt in ("fp16", "bf16"):
        c = nrc.Cache(dtype=dt, width=128, hidden_layers=7, seed=2106)
        c.set_state(w128)
        got = c.infer(sample).cpu().numpy().astype(np.float64)
        err = np.abs(got - ref128) / np.maximum(np.abs(ref128), tau128)
        for k in range(3):
            c.infer(queries[k % 2], rgb)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(frames)]
        for k, e in enumerate(ev):
            flush.zero_()
            e[0].record(st)
            c.infer(queries[k % 2], rgb)
            e[1].record(st)
        torch.cuda.synchronize()
        c.check_error()
        ms = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        tf = FLOP_QUERY_W128 * N_QUERIES / (ms / 1e3) / 1e12
        out[f"{dt}_width128_7hidden"] = {"infer_ms": ms, "tflops": tf, "frac_of_peak": tf / burst,
                                         "err_median": float(np.median(err)), "err_max": float(err.max())}
        c.close()
    out["workload"] = ("1080p query batch per dtype (FP32: SIMT parity path; width 128: plain per-layer FP32 path "
                       "and the tensor-core FP16 / BF16 kernel); error against the FP32 path of the same width on "
                       "2,000 queries")
    return out


def run_paths(dtype: str, flush, frames: int = 20):
    """A 1080p frame through the training-record pipeline (Sec. 3.3-3.5, the
    termination heuristic of Eqs. 3-4): terminate every pixel's path and pick
    the training paths, query the cache at the terminal vertices and at the
    training paths' tails, build the self-training records, train 4 steps of
    16,384 records on them and composite the pixels.  The tail queries sit
    after the render queries in one buffer, so one query launch answers both.
    The tile side is adapted during the warm-up frames toward 65,536 training
    records and then held; each stage is timed with CUDA events."""
    import numpy as np
    import torch

    from paper_2106_12372_gb300 import nrc, synth

    dev = torch.device("cuda:0")
    W, H, K, rep = 1920, 1080, 10, 4
    # synthetic cube-room paths of a 480 x 270 view, tiled 4 x 4 across the
    # 1080p frame (the same work per pixel; generating 2 M paths on the host
    # takes about half a minute)
    v = torch.from_numpy(synth.make_paths(W // rep, H // rep, K, seed=2106 + 3)).to(dev)
    v = v.view(H // rep, W // rep, K, 24).repeat(rep, rep, 1, 1).reshape(W * H, K, 24).contiguous()
    cache = nrc.Cache(dtype=dtype, seed=2106)
    cam = synth.PATH_CAMERA
    P = W * H
    em = torch.empty((P, 3), device=dev)
    tp = torch.empty((P, 3), device=dev)
    img = torch.empty((P, 3), device=dev)
    pool = torch.zeros((N_POOL, 16), device=dev)
    tg = torch.zeros((N_POOL, 3), device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    tile, gen = 4, []
    for f in range(8):  # warm-up: adapt the tile side toward N_POOL records
        prm = nrc.PathParams(0.01, tile, f % tile, (3 * f) % tile, f % 16, 0.8)
        _, _, _, tiles, tq = nrc.paths_terminate(v, W, H, cam, prm)
        tail = cache.infer(tq)
        pool_, tg_, cnt = nrc.paths_records(v, W, H, cam, prm, tiles, tail, N_POOL)
        n = int(cnt.item())
        gen.append(n)
        tile = nrc.paths_adapt_tile(tile, n, N_POOL)
    nt = nrc.paths_tile_count(W, H, tile)
    tiles = torch.empty((nt, 4), dtype=torch.int32, device=dev)
    # the tail queries follow the render queries in one buffer: one query launch answers both
    q_all = torch.zeros((P + nt, 16), device=dev)
    rgb_all = torch.empty((P + nt, 3), device=dev)
    rq, tq = q_all[:P], q_all[P:]
    rgb, tail = rgb_all[:P], rgb_all[P:]
    offsets = torch.empty(nrc.paths_offsets_count(nt), dtype=torch.int64, device=dev)
    st = torch.cuda.current_stream()
    names = ("terminate", "queries", "records", "train", "composite")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(frames + 3)]
    counts = torch.zeros(frames + 3, dtype=torch.int64, device=dev)
    for f, e in enumerate(ev):
        prm = nrc.PathParams(0.01, tile, f % tile, (5 * f) % tile, f % 16, 0.8)
        flush.zero_()
        e[0].record(st)
        nrc.paths_terminate(v, W, H, cam, prm, out=(rq, em, tp, tiles, tq))
        e[1].record(st)
        cache.infer(q_all, rgb_all)
        e[2].record(st)
        nrc.paths_records(v, W, H, cam, prm, tiles, tail, N_POOL, out=(pool, tg, offsets, count))
        e[3].record(st)
        cache.frame(rq[:0], rgb[:0], pool, tg, BATCH, N_STEPS, synth.frame_seed(2106 + 3, f))
        e[4].record(st)
        nrc.paths_composite(em, tp, rgb, out=img)
        e[5].record(st)
        counts[f] = count[0]
    torch.cuda.synchronize()
    cache.check_error()
    ev = ev[3:]
    out = {k: float(np.median([e[i].elapsed_time(e[i + 1]) for e in ev])) for i, k in enumerate(names)}
    out = {k + "_ms": v_ for k, v_ in out.items()}
    total = float(np.median([e[0].elapsed_time(e[-1]) for e in ev]))
    out.update(frame_ms=total, mqueries_per_s=(P + nt) / (total / 1e3) / 1e6, tile=tile, training_paths=nt,
               records_per_frame_median=int(np.median(counts.cpu().numpy()[3:])), warmup_records=gen,
               workload=("1080p frame, 10-vertex synthetic cube-room paths (a 480x270 path set tiled 4x4), "
                         "c = 0.01, roulette suffix every 16th tile (q = 0.8), tile adapted to ~65,536 records, "
                         "4 x 16,384 training steps on the first 65,536 records"))
    cache.close()
    return out


SMALL_Q, SMALL_B = 65536, 16384


def run_small(flush, frames: int = 20):
    """The small configuration: 65,536 queries and one training step of
    16,384 records from a 16,384-record pool, in FP32, on the fused (SIMT)
    path and on the plain per-layer path; ms per frame (median)."""
    import numpy as np
    import torch

    from paper_2106_12372_gb300 import nrc, synth

    dev = torch.device("cuda:0")
    q = torch.from_numpy(synth.make_records(SMALL_Q, seed=2107)).to(dev)
    pool, tgt = (torch.from_numpy(x).to(dev) for x in synth.make_training_pool(SMALL_B, seed=2108))
    rgb = torch.empty((SMALL_Q, 3), device=dev)
    st = torch.cuda.current_stream()
    out = {}
    for name, path in (("fused_fp32", nrc.PATH_FUSED), ("plain_fp32", nrc.PATH_PLAIN)):
        c = nrc.Cache(dtype="fp32", path=path, seed=2107)
        for k in range(3):
            c.frame(q, rgb, pool, tgt, SMALL_B, 1, synth.frame_seed(2107, k))
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(frames)]
        for k, e in enumerate(ev):
            flush.zero_()
            e[0].record(st)
            c.frame(q, rgb, pool, tgt, SMALL_B, 1, synth.frame_seed(2107, 3 + k))
            e[1].record(st)
        torch.cuda.synchronize()
        c.check_error()
        out[name + "_ms"] = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        c.close()
    out["workload"] = "65,536 queries + 1 step of 16,384 records from a 16,384-record pool, FP32"
    return out


def cpu_oracle_small(seed: int = 2107):
    """The FP64 oracle on one whole small-configuration frame (ms, cores)."""
    from oracle import oracle as O
    from paper_2106_12372_gb300 import synth

    dims = synth.layer_dims()
    q = synth.make_records(SMALL_Q, seed=seed)
    pool, tgt = synth.make_training_pool(SMALL_B, seed=seed + 1)
    st = O.TrainState(synth.xavier_weights(dims, seed=seed), dims)
    O.infer(st.W, dims, q[:1024])  # load the library and its threads
    t0 = time.perf_counter()
    O.infer(st.W, dims, q)
    st.step(pool, tgt, SMALL_B, synth.frame_seed(seed, 0), 0)
    return (time.perf_counter() - t0) * 1e3, int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


def run_serving(queries, dtype: str, seconds: float, rate_scale: float = 1.0):
    """Eight viewports (4 x 1920x1080, 4 x 3840x2160) with Poisson frame
    arrivals at 30-120 Hz each (rates seeded; all multiplied by rate_scale
    for the load sweep), served by the continuous-
    batching server under a 16 GB memory budget; each frame is a cache query
    for every pixel plus 4 training steps of 16,384 records from the
    viewport's resident 65,536-record pool.  Latency runs from the frame's
    scheduled arrival to the host callback at the end of its batch."""
    import numpy as np
    import torch

    from paper_2106_12372_gb300 import nrc, synth

    srv = nrc.Server(nrc.default_config(dtype=dtype))
    rng = np.random.default_rng(2106 + 5)
    sizes = [1920 * 1080] * 4 + [3840 * 2160] * 4
    vps = []
    for v, n in enumerate(sizes):
        vid = srv.open_viewport(n, N_POOL, n_slots=2, seed=2106 + 500 + v)
        pool, tgt, _ = srv.pool(vid)
        p, t = synth.make_training_pool(N_POOL, seed=2106 + 500 + v)
        pool.copy_(torch.from_numpy(p))
        tgt.copy_(torch.from_numpy(t))
        for slot in range(2):
            r, _, _ = srv.buffers(vid, slot)
            for j in range(n // N_QUERIES):
                r[j * N_QUERIES:(j + 1) * N_QUERIES].copy_(queries[(j + slot) % 2])
        vps.append((vid, n, float(rng.uniform(30.0, 120.0)) * rate_scale))
    torch.cuda.synchronize()
    info0 = srv.info()
    # warm-up: two frames per viewport
    def wait_slot(t_end):
        if time.monotonic() > t_end:
            raise RuntimeError("serving: a frame slot stayed busy for 30 s")

    for f in range(2):
        for vid, n, _ in vps:
            t_end = time.monotonic() + 30.0
            while not srv.submit(vid, f % 2, n, synth.frame_seed(vid, f)):
                wait_slot(t_end)
                srv.poll(timeout_ms=5)
    srv.drain()
    srv.poll(max_out=4096)
    arrivals = []
    for vid, n, rate in vps:
        t = rng.exponential(1.0 / rate)
        while t < seconds:
            arrivals.append((t, vid, n))
            t += rng.exponential(1.0 / rate)
    arrivals.sort()
    nxt = {vid: 2 for vid, _, _ in vps}
    done = []
    t0 = nrc.now_ns() + 1_000_000
    for t, vid, n in arrivals:
        due = t0 + int(t * 1e9)
        while nrc.now_ns() < due:
            done += srv.poll(timeout_ms=0)
            if due - nrc.now_ns() > 300_000:
                time.sleep(0.0001)
        f = nxt[vid]
        t_end = time.monotonic() + 30.0
        while not srv.submit(vid, f % 2, n, synth.frame_seed(vid, f), arrival_ns=due, tag=f):
            wait_slot(t_end)
            done += srv.poll(timeout_ms=1)
        nxt[vid] += 1
    srv.drain()
    done += srv.poll(max_out=65536)
    info = srv.info()
    srv.close()
    lat = np.array([(d.done_ns - d.arrival_ns) / 1e6 for d in done])
    span = (max(d.done_ns for d in done) - t0) / 1e9
    q = sum(d.n_queries for d in done)
    offered = sum(rate * n for _, n, rate in vps)
    return {
        "workload": "8 viewports (4 x 1920x1080, 4 x 3840x2160), Poisson arrivals 30-120 Hz each, per frame all "
                    "pixels queried + 4 x 16,384-record training steps; 16 GB admission budget",
        "seconds": seconds, "rate_scale": rate_scale, "frames": len(done), "failed": int(sum(d.failed for d in done)),
        "p50_frame_ms": float(np.percentile(lat, 50)), "p99_frame_ms": float(np.percentile(lat, 99)),
        "max_frame_ms": float(lat.max()), "mean_batch_frames": float(np.mean([d.batch_frames for d in done])),
        "aggregate_mqueries_per_s": q / span / 1e6, "offered_mqueries_per_s": offered / 1e6,
        "rates_hz": [round(r, 1) for _, _, r in vps], "resident_gb": info0.memory_used / 1e9,
        "batches": int(info.batches),
    }


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2106_12372_gb300 import nrc, synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2106_12372_gb300 import build

    # one process compiles (if the library is stale); the other ranks then find it built
    if not build_once(ws, rank, build.build):
        raise SystemExit("bench.py: the CUDA library failed to build on rank 0")
    stream = torch.cuda.current_stream()

    seed = 2106 + rank
    queries = [torch.from_numpy(synth.make_records(N_QUERIES, seed=seed + k)).to(dev) for k in range(2)]
    pool_np, tgt_np = synth.make_training_pool(N_POOL, seed=seed)
    pool, tgt = torch.from_numpy(pool_np).to(dev), torch.from_numpy(tgt_np).to(dev)
    rgb = torch.empty((N_QUERIES, 3), device=dev)
    losses = torch.zeros(N_STEPS, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # 256 MB > 129 MB L2

    cache = nrc.Cache(dtype=args.dtype, seed=seed)

    empty_q = queries[0][:0]

    def frame(k, ev=None):
        # the frame through the C ABI: one nrc_frame call answers the frame's
        # queries (weights from before its training) and runs its N_STEPS
        # training steps -- one persistent launch on the 16-bit caches
        if ev:
            ev[0].record(stream)
        cache.frame(queries[k % 2], rgb, pool, tgt, BATCH, N_STEPS, synth.frame_seed(seed, k), loss_out=losses)
        if ev:
            ev[1].record(stream)

    for k in range(args.warmup):
        frame(k)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    launches0 = cache.launches
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # untimed frames for 0.3 s right before the timed region, so that the
        # clock record holds samples under this load whatever --steps is
        t_burn = time.perf_counter()
        kb = 0
        while time.perf_counter() - t_burn < 0.3:
            for _ in range(50):
                frame(args.warmup + kb)
                kb += 1
            torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            frame(args.warmup + k, evs[k])
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = cache.launches - launches0 - kb * (1 if args.dtype != "fp32" else 0)
    cache.check_error()
    frame_ms = [e[0].elapsed_time(e[1]) for e in evs]
    total_ms, value = job_throughput(sum(frame_ms), N_QUERIES, args.steps, ws, device=dev)
    split_ctas = cache.frame_ctas(N_QUERIES, BATCH, N_STEPS)

    # breakdown (not the headline): the same frame's queries alone (nrc_infer)
    # and its training alone, as the fused training-only launch and as
    # separate gradient + Adam launches
    def timed(fn, n=20):
        e = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n)]
        for i in range(n):
            flush.zero_()
            e[i][0].record(stream)
            fn(i)
            e[i][1].record(stream)
        torch.cuda.synchronize()
        return statistics.median(x[0].elapsed_time(x[1]) for x in e)

    w_keep = cache.get_state()
    infer_ms = timed(lambda i: cache.infer(queries[i % 2], rgb))
    train_fused_ms = timed(lambda i: cache.frame(empty_q, rgb, pool, tgt, BATCH, N_STEPS, synth.frame_seed(seed, i)))
    cache.set_frame_ctas(-1)
    train_sep_ms = timed(lambda i: cache.frame(empty_q, rgb, pool, tgt, BATCH, N_STEPS, synth.frame_seed(seed, i)))
    seq_frame_ms = timed(lambda i: cache.frame(queries[i % 2], rgb, pool, tgt, BATCH, N_STEPS, synth.frame_seed(seed, i)))
    cache.set_frame_ctas(0)
    cache.set_state(w_keep[0], w_keep[1], w_keep[2], w_keep[3])

    # plain per-layer FP32 path on the same frame (a few frames; same cache shape)
    plain = nrc.Cache(dtype="fp32", path=nrc.PATH_PLAIN, seed=seed)
    pev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    plain_ms = []
    for k in range(3):
        flush.zero_()
        pev[0].record(stream)
        plain.infer(queries[0], rgb)
        plain.frame(empty_q, rgb, pool, tgt, BATCH, N_STEPS, synth.frame_seed(seed, k))
        pev[1].record(stream)
        torch.cuda.synchronize()
        if k > 0:
            plain_ms.append(pev[0].elapsed_time(pev[1]))
    plain.close()

    batched = serving = serving_sweep = shampoo = precision = paths = small = None
    if not args.no_extras and ws == 1 and args.dtype != "fp32":
        batched = run_batched(queries, args.dtype, 30, flush)
        serving = run_serving(queries, args.dtype, args.serve_seconds)
        # the same viewports at 1x .. 8x their frame rates: toward saturation, where continuous batching
        # merges frames (mean_batch_frames > 1)
        keys = ("rate_scale", "offered_mqueries_per_s", "aggregate_mqueries_per_s", "p50_frame_ms", "p99_frame_ms",
                "max_frame_ms", "mean_batch_frames", "frames", "failed")
        serving_sweep = [{k: r[k] for k in keys} for r in
                         (run_serving(queries, args.dtype, args.sweep_seconds, sc) for sc in (1.0, 2.0, 4.0, 8.0))]
        shampoo = run_shampoo(pool, tgt, args.dtype, 30, flush)
        precision = run_precision(queries, flush)
        paths = run_paths(args.dtype, flush)
        small = run_small(flush)

    # end to end: host (pinned) buffers through nrc_frame_host, copies inside the timed region
    qh = torch.from_numpy(synth.make_records(N_QUERIES, seed=seed + 7)).pin_memory()
    ph, th = pool.cpu().pin_memory(), tgt.cpu().pin_memory()
    rgb_h = torch.empty((N_QUERIES, 3)).pin_memory()
    loss_h = torch.zeros(N_STEPS).pin_memory()
    for k in range(2):
        cache.frame_host(qh, rgb_h, ph, th, BATCH, N_STEPS, synth.frame_seed(seed, k), loss_out=loss_h)
    e2e_n = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_n):
        cache.frame_host(qh, rgb_h, ph, th, BATCH, N_STEPS, synth.frame_seed(seed, k), loss_out=loss_h)
    e2e_s = (time.perf_counter() - t0) / e2e_n
    h2d = N_QUERIES * 64 + N_POOL * 64 + N_POOL * 12
    d2h = N_QUERIES * 12 + N_STEPS * 4

    if rank != 0:
        return
    burst, sustained, hbm, src = peaks()
    frame_flop = FLOP_QUERY * N_QUERIES + FLOP_RECORD * BATCH * N_STEPS
    med = statistics.median(frame_ms)
    achieved = frame_flop / (med / 1e3) / 1e12
    p99 = float(np.percentile(frame_ms, 99))
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        v, d, cores, _ = cpu_oracle_frame(args.cpu_budget)
        cpu = {"value": v, "unit": "Mqueries/s", "cores": cores, "kind": "oracle", "sample": d}
        if small is not None:
            small["oracle_fp64_ms"], small["oracle_cores"] = cpu_oracle_small()
    clocks = clk.summary()
    clocks["window"] = "0.3 s of untimed frames right before the timed frames, then the timed frames"
    line = {
        "metric": METRIC, "value": value, "unit": "Mqueries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "queries": N_QUERIES, "train_steps": N_STEPS, "batch": BATCH,
                   "pool": N_POOL, "l2": "flushed (256 MB write) between frames, outside the events",
                   "parallelism": f"replicas x{ws}"},
        "frame_ms_median": med, "frame_ms_p99": p99, "frame_train_ctas": split_ctas,
        "breakdown": {"queries_alone_ms": infer_ms, "train_alone_fused_ms": train_fused_ms,
                      "train_alone_separate_launches_ms": train_sep_ms,
                      "frame_as_separate_launches_ms": seq_frame_ms,
                      "note": "medians of 20 frames each, L2 flushed; the headline frame is one fused launch"},
        "frame_tflops": frame_flop / (med / 1e3) / 1e12, "frame_frac_of_peak": frame_flop / (med / 1e3) / 1e12 / burst,
        "plain_fp32_ms_per_frame": statistics.median(plain_ms) if plain_ms else None,
        "batched_caches": batched,
        "serving": serving,
        "serving_sweep": serving_sweep,
        "shampoo": shampoo,
        "precision": precision,
        "paths": paths,
        "small_config": small,
        "roofline": {"kernel": "k_frame_tc (the whole frame: queries + 4 training steps, one launch)",
                     "bound": "tensor", "achieved": achieved,
                     "peak": burst, "unit": "TFLOP/s", "frac": achieved / burst, "traffic": frame_traffic(),
                     "peak_source": f"{src} bf16 dense burst (fp16 peak = bf16 peak)"},
        "cpu_baseline": cpu,
        "e2e": {"value": N_QUERIES / e2e_s / 1e6, "unit": "Mqueries/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3},
        "gpu_launches": launches,
        "clocks": clocks,
        "frame_ms_x_sm_ghz": (med * clocks["sm_mhz"] / 1e3) if clocks.get("sm_mhz") else None,
        "paper_context": "RTX 3090, half: query 1.59 ms + training 1.11 ms per 1080p frame (Table 3)",
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nrc", choices=["nrc", "reference"])
    ap.add_argument("--dtype", default="fp16", choices=["fp16", "bf16", "fp32"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched-caches and serving measurements")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--sweep-seconds", type=float, default=2.0, help="arrivals per point of the serving load sweep")
    ap.add_argument("--ref-seconds", type=float, default=90.0, help="oracle work of the whole --impl reference run")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
