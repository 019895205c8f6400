"""Writes grouped_shapes_seed1.json: the 64 independent convolution problems of
the grouped-launch workload, drawn once with numpy.random.default_rng(1).

Per problem: N in {1..16}, C and K in {16, 32, ..., 512}, H = W in
{7, 14, 28, 56, 112}, R = S in {1, 3, 5, 7}, stride in {1, 2}, pad = R // 2,
dilation 1. The drawn list is committed so that later numpy versions cannot
change it. This script calls nothing but numpy.
"""
import json
import os

import numpy as np


def main():
    rng = np.random.default_rng(1)
    probs = []
    for _ in range(64):
        n = int(rng.integers(1, 17))
        c = 16 * int(rng.integers(1, 33))
        k = 16 * int(rng.integers(1, 33))
        hw = int(rng.choice([7, 14, 28, 56, 112]))
        r = int(rng.choice([1, 3, 5, 7]))
        st = int(rng.choice([1, 2]))
        probs.append(dict(N=n, C=c, H=hw, W=hw, K=k, R=r, S=r, stride=st, pad=r // 2))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grouped_shapes_seed1.json")
    with open(out, "w") as f:
        json.dump({"source": "numpy.random.default_rng(1), see make_grouped_shapes.py",
                   "problems": probs}, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
