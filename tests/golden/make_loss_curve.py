"""Writes tests/golden/loss_curve_fp64.json: the FP64 oracle's training-loss curve.

1000 optimisation steps = 250 frames x 4 steps (Sec. 3.3: several steps per
frame on disjoint slices of the frame's shuffled records; Sec. 3.5: s = 4
batches of l = 16,384 records), Adam lr 1e-2, beta (0.9, 0.99), relative L2
loss with eps = 0.01 (Eq. 5), pad value 1, cheap encoding.  Each frame draws a
fresh 65,536-record pool from the seeded generator.  Calls only the oracle.

    python tests/golden/make_loss_curve.py
"""
import json
import os
import sys
import time

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
    dims = synth.layer_dims()
    st = O.TrainState(synth.xavier_weights(dims, seed=SEED), dims)
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
           "loss": losses}
    json.dump(out, open(os.path.join(HERE, "loss_curve_fp64.json"), "w"), indent=0)


if __name__ == "__main__":
    main()
