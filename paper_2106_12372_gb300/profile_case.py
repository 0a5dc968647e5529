"""Runs one hot-path stage on seeded inputs for profiling (ncu / nsight) on cuda:0.

    python -m paper_2106_12372_gb300.profile_case --what infer --n 2073600 --dtype fp16 --iters 3
    python -m paper_2106_12372_gb300.profile_case --what train --batch 16384 --dtype fp16 --iters 3
"""
from __future__ import annotations

import argparse

import torch

from paper_2106_12372_gb300 import build, nrc, synth


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", choices=["infer", "train", "frame"], default="infer")
    ap.add_argument("--n", type=int, default=1920 * 1080)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--dtype", default="fp16")
    ap.add_argument("--iters", type=int, default=3)
    args = ap.parse_args()
    build.build()
    dev = torch.device("cuda:0")
    cache = nrc.Cache(dtype=args.dtype)
    pool_np, tgt_np = synth.make_training_pool(args.batch * args.steps, seed=5)
    pool, tgt = torch.from_numpy(pool_np).to(dev), torch.from_numpy(tgt_np).to(dev)
    rec = torch.from_numpy(synth.make_records(args.n, seed=6)).to(dev) if args.what != "train" else None
    rgb = torch.empty((args.n, 3), device=dev) if rec is not None else None
    for it in range(args.iters):
        if args.what in ("infer", "frame"):
            cache.infer(rec, rgb)
        if args.what in ("train", "frame"):
            for s in range(args.steps):
                cache.train_step(pool, tgt, args.batch, synth.frame_seed(5, it), s)
    torch.cuda.synchronize()
    cache.check_error()
    print("ok")


if __name__ == "__main__":
    main()
