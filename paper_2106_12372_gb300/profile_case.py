"""Runs one hot-path stage on seeded inputs for profiling (ncu / nsight) on cuda:0.

    python -m paper_2106_12372_gb300.profile_case --what infer --n 2073600 --dtype fp16 --iters 3
    python -m paper_2106_12372_gb300.profile_case --what train --batch 16384 --dtype fp16 --iters 3
    python -m paper_2106_12372_gb300.profile_case --what frame --n 2073600 --steps 4 --iters 3
    python -m paper_2106_12372_gb300.profile_case --what train-fused --batch 16384 --steps 4 --ctas 43 --iters 3
    python -m paper_2106_12372_gb300.profile_case --what infer --net-width 128 --hidden 7 --dtype fp16
    python -m paper_2106_12372_gb300.profile_case --what paths --width 1920 --height 1080 --iters 3

``train-fused`` runs a frame without queries through the frame kernel's
training role on --ctas CTAs (a frame without queries otherwise takes the
separate gradient and Adam launches).  ``paths`` runs the training-record pipeline around the query (terminate, the
render and tail queries, the self-training records, 4 training steps, the
composite) on synthetic 10-vertex paths: a quarter-resolution path set tiled
4 x 4 over the frame, training tiles of 8 x 8 pixels.
"""
from __future__ import annotations

import argparse

import torch

from paper_2106_12372_gb300 import build, nrc, synth


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", choices=["infer", "train", "train-fused", "frame", "paths"], default="infer")
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--n", type=int, default=1920 * 1080)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--dtype", default="fp16")
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--net-width", type=int, default=64, help="64, or 128 (with --hidden 7) for the wide network")
    ap.add_argument("--hidden", type=int, default=5)
    ap.add_argument("--ctas", type=int, default=43, help="training CTAs of --what train-fused")
    args = ap.parse_args()
    build.build()
    dev = torch.device("cuda:0")
    if args.what == "paths":
        run_paths(args, dev)
        return
    cache = nrc.Cache(dtype=args.dtype, width=args.net_width, hidden_layers=args.hidden)
    pool_np, tgt_np = synth.make_training_pool(args.batch * args.steps, seed=5)
    pool, tgt = torch.from_numpy(pool_np).to(dev), torch.from_numpy(tgt_np).to(dev)
    rec = torch.from_numpy(synth.make_records(args.n, seed=6)).to(dev) if not args.what.startswith("train") else None
    rgb = torch.empty((args.n, 3), device=dev) if rec is not None else None
    if args.what == "train-fused":
        cache.set_frame_ctas(args.ctas)
        q0 = torch.zeros((1, 16), device=dev)
        rec, rgb = q0[:0], q0[:0, :3]
    for it in range(args.iters):
        if args.what in ("frame", "train-fused"):  # the fused frame: one launch of queries and training steps
            cache.frame(rec, rgb, pool, tgt, args.batch, args.steps, synth.frame_seed(5, it))
        if args.what == "infer":
            cache.infer(rec, rgb)
        if args.what == "train":
            for s in range(args.steps):
                cache.train_step(pool, tgt, args.batch, synth.frame_seed(5, it), s)
    torch.cuda.synchronize()
    cache.check_error()
    print("ok")


def run_paths(args, dev) -> None:
    W, H, K, rep = args.width, args.height, 10, 4
    if W % rep or H % rep:
        raise SystemExit("--width and --height must be multiples of 4")
    v = torch.from_numpy(synth.make_paths(W // rep, H // rep, K, seed=2109)).to(dev)
    v = v.view(H // rep, W // rep, K, 24).repeat(rep, rep, 1, 1).reshape(W * H, K, 24).contiguous()
    cache = nrc.Cache(dtype=args.dtype)
    cam = synth.PATH_CAMERA
    rgb = torch.empty((W * H, 3), device=dev)
    for it in range(args.iters):
        prm = nrc.PathParams(0.01, 8, it % 8, (3 * it) % 8, it % 16, 0.8)
        rq, em, tp, tiles, tq = nrc.paths_terminate(v, W, H, cam, prm)
        cache.infer(rq, rgb)
        tail = cache.infer(tq)
        pool, tg, count = nrc.paths_records(v, W, H, cam, prm, tiles, tail, args.batch * args.steps)
        cache.frame(rq[:0], rgb[:0], pool, tg, args.batch, args.steps, synth.frame_seed(2109, it))
        nrc.paths_composite(em, tp, rgb)
    torch.cuda.synchronize()
    cache.check_error()
    print("ok")


if __name__ == "__main__":
    main()
