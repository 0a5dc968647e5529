"""Writes tests/golden/width128_curve_fp64.json: the FP64 oracle's 100-step
training-loss curves of the width-128, 7-hidden-layer network in four
realizations.

The run is the one tests/test_gpu_width128.py makes on the GPU: Xavier weights
from seed 56, a 4 x 2,048-record pool from seed 57, 25 frames of 4 steps of
2,048 records (frame seeds from 58), Adam lr 1e-2, beta (0.9, 0.99), relative
L2 loss with eps = 0.01 (Eq. 5), pad value 1, cheap encoding.  Realization
k >= 1 starts from the same weights multiplied by (1 + 1e-7 z), z ~ N(0, 1)
from numpy's generator seeded with k: independent runs of the same chaotic
training process, whose spread is the loss-curve test's tolerance.  Calls
only the oracle.

    python tests/golden/make_width128_curve.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2106_12372_gb300 import synth  # noqa: E402

REALIZATIONS = 4


def main():
    dims = synth.layer_dims(width=128, hidden_layers=7)
    w0 = synth.xavier_weights(dims, seed=56).astype(np.float64)
    pool, tgt = synth.make_training_pool(4 * 2048, seed=57)
    curves = []
    for k in range(REALIZATIONS):
        w = w0 if k == 0 else w0 * (1.0 + 1e-7 * np.random.default_rng(k).standard_normal(w0.size))
        st = O.TrainState(w, dims)
        curves.append([st.step(pool, tgt, 2048, synth.frame_seed(58, f), s) for f in range(25) for s in range(4)])
        print("realization", k, "100-step median", float(np.median(curves[-1])), flush=True)
    out = {"what": "FP64 oracle loss curves, width 128, 7 hidden layers, 100 steps of 2,048 records",
           "realizations": curves, "medians": [float(np.median(c)) for c in curves]}
    json.dump(out, open(os.path.join(HERE, "width128_curve_fp64.json"), "w"))


if __name__ == "__main__":
    main()
