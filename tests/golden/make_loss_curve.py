"""Writes tests/golden/loss_curve_fp64.json: the FP64 oracle's training-loss curve.

1000 optimisation steps = 250 frames x 4 steps (Sec. 3.3: several steps per
frame on disjoint slices of the frame's shuffled records; Sec. 3.5: s = 4
batches of l = 16,384 records), Adam lr 1e-2, beta (0.9, 0.99), relative L2
loss with eps = 0.01 (Eq. 5), pad value 1, cheap encoding.  Each frame draws a
fresh 65,536-record pool from the seeded generator.  Calls only the oracle.

    python tests/golden/make_loss_curve.py                 # loss_curve_fp64.json
    python tests/golden/make_loss_curve.py --realization 1  # loss_curve_fp64_r1.json

Realization k >= 1 starts from the same weights multiplied by (1 + 1e-7 z),
z ~ N(0, 1) from numpy's generator seeded with k: an independent run of the
same chaotic training process, which measures how far two faithful runs of
the method drift apart (the tolerance of the loss-curve test).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2106_12372_gb300 import synth  # noqa: E402

SEED = 2110
FRAMES = 250
STEPS = 4
BATCH = 16384


def pool_for(frame):
    return synth.make_training_pool(BATCH * STEPS, seed=SEED * 1000 + frame)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--realization", type=int, default=0)
    k = ap.parse_args().realization
    dims = synth.layer_dims()
    w0 = synth.xavier_weights(dims, seed=SEED).astype(np.float64)
    if k > 0:
        w0 = w0 * (1.0 + 1e-7 * np.random.default_rng(k).standard_normal(w0.size))
    st = O.TrainState(w0, dims)
    losses = []
    t0 = time.time()
    for f in range(FRAMES):
        pool, tgt = pool_for(f)
        fs = synth.frame_seed(SEED, f)
        for s in range(STEPS):
            losses.append(st.step(pool, tgt, BATCH, fs, s))
        if f % 25 == 0:
            print(f"frame {f} loss {losses[-1]:.5f} ({time.time() - t0:.0f} s)", flush=True)
    out = {"_source": "FP64 oracle (oracle/nrc_oracle.cpp) via tests/golden/make_loss_curve.py; "
                      "Sec. 3.3 / 3.5 schedule, Eq. 5 loss, Adam (Sec. 5)",
           "seed": SEED, "frames": FRAMES, "steps_per_frame": STEPS, "batch": BATCH, "pool": BATCH * STEPS,
           "pool_seed": "SEED * 1000 + frame", "frame_seed": "synth.frame_seed(SEED, frame)",
           "realization": k, "loss": losses}
    name = "loss_curve_fp64.json" if k == 0 else f"loss_curve_fp64_r{k}.json"
    json.dump(out, open(os.path.join(HERE, name), "w"), indent=0)


if __name__ == "__main__":
    main()
