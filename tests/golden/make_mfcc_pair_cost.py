"""Writes mfcc_pair_60000x75000.txt: the optimal cost D* of the orchestral-length
MFCC-like pair (60000 x 64-d frames against a 75000-frame warp plus noise), as
oracle 2 (Algorithm 2, FP64 cost and accumulation) returns it.

The pair is too large for a test to run the oracle on it (about 4.5e9 cells,
several minutes on one core), so its cost is stored once.  Only the seeded input
generator and the oracle are called here.

    python tests/golden/make_mfcc_pair_cost.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2008_02734_b300 import synth  # noqa: E402

OUT = os.path.join(HERE, "mfcc_pair_60000x75000.txt")


def main():
    X, Y = synth.workload_precision()
    t = time.perf_counter()
    path, cost, cells = oracle.linmdtw(X, Y)
    dt = time.perf_counter() - t
    with open(OUT, "w") as f:
        f.write("# Optimal cost of synth.workload_precision() (60000 x 75000, d = 64), oracle 2\n")
        f.write("# (Algorithm 2 with FP64 Euclidean cost and FP64 accumulation, base case m = 500).\n")
        f.write(f"# Written by tests/golden/make_mfcc_pair_cost.py in {dt:.0f} s on one core.\n")
        f.write("# fields: M|N|d|cost (repr of the FP64 value)|path length|processed cells\n")
        f.write(f"{len(X)}|{len(Y)}|{X.shape[1]}|{cost!r}|{len(path)}|{cells}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
