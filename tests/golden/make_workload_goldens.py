"""Writes the stored oracle results of the full-size workloads that the GPU
tests check but cannot afford to run the oracle on at test time:

* batch_chroma_256.txt -- oracle 1's optimal cost (FP64) of every pair of the
  uneven batch synth.workload_batch() (256 chroma-like d=12 pairs, M and N in
  [1000, 20000]);
* batch_int_256.txt    -- oracle 1's cost (int64) and canonical path (its length
  and the SHA-256 of its int32 (K, 2) little-endian bytes) of every pair of
  synth.workload_batch_int() (the same shapes, int32 |x-y| data);
* edit_20000.txt       -- the edit oracle's cost and canonical node path (length,
  SHA-256) of synth.workload_edit_pair() (unit costs);
* local_20000x24000.txt -- the local-alignment oracle's score, start and end
  nodes and node path (length, SHA-256) of synth.workload_local_pair() (scores
  +2 / -3 / -3).

Only the seeded input generators and oracle/ are called.  The batch pairs run
one per process (spawned) on every host core; about a minute on 8 cores.

    python tests/golden/make_workload_goldens.py
"""
import hashlib
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2008_02734_b300 import synth  # noqa: E402

B = 256


def path_sha256(path) -> str:
    return hashlib.sha256(np.ascontiguousarray(path, dtype="<i4").tobytes()).hexdigest()


def _chroma(k):
    X, Y = synth.batch_pair(k)
    return k, len(X), len(Y), oracle.dtw(X, Y)[1]


def _int(k):
    X, Y = synth.batch_int_pair(k)
    p, c = oracle.dtw(X, Y)
    return k, len(X), len(Y), c, len(p), path_sha256(p)


def main():
    oracle.build()
    ctx = mp.get_context("spawn")
    n = os.cpu_count() or 1
    t = time.perf_counter()
    with ctx.Pool(n) as pool:
        # largest pairs first, so that no long pair starts last
        M, N = synth.workload_batch_sizes()
        order = sorted(range(B), key=lambda k: -int(M[k]) * int(N[k]))
        chroma = sorted(pool.map(_chroma, order, chunksize=1))
        ints = sorted(pool.map(_int, order, chunksize=1))
    dt = time.perf_counter() - t
    with open(os.path.join(HERE, "batch_chroma_256.txt"), "w") as f:
        f.write("# Oracle 1 (FP64 textbook DTW) on synth.workload_batch(): 256 chroma-like d=12 pairs.\n")
        f.write(f"# Written by tests/golden/make_workload_goldens.py ({dt:.0f} s for both batches on {n} cores).\n")
        f.write("# fields: pair|M|N|cost (repr of the FP64 value)\n")
        for k, m, nn, c in chroma:
            f.write(f"{k}|{m}|{nn}|{c!r}\n")
    with open(os.path.join(HERE, "batch_int_256.txt"), "w") as f:
        f.write("# Oracle 1 (int64 textbook DTW, ties DIAG > UP > LEFT) on synth.workload_batch_int().\n")
        f.write("# Written by tests/golden/make_workload_goldens.py.\n")
        f.write("# fields: pair|M|N|cost|path length|sha256 of the int32 (K, 2) path bytes\n")
        for k, m, nn, c, K, h in ints:
            f.write(f"{k}|{m}|{nn}|{c}|{K}|{h}\n")

    X, Y = synth.workload_edit_pair()
    t = time.perf_counter()
    p, c = oracle.edit(X, Y)
    dt = time.perf_counter() - t
    with open(os.path.join(HERE, "edit_20000.txt"), "w") as f:
        f.write("# Edit oracle (unit costs, ties DIAG > UP > LEFT) on synth.workload_edit_pair().\n")
        f.write(f"# Written by tests/golden/make_workload_goldens.py ({dt:.1f} s on one core).\n")
        f.write("# fields: M|N|cost|node path length|sha256 of the int32 (K, 2) node path bytes\n")
        f.write(f"{len(X)}|{len(Y)}|{c}|{len(p)}|{path_sha256(p)}\n")

    X, Y = synth.workload_local_pair()
    t = time.perf_counter()
    p, s, se = oracle.local(X, Y, match=2, mismatch=3, gap=3)
    dt = time.perf_counter() - t
    with open(os.path.join(HERE, "local_20000x24000.txt"), "w") as f:
        f.write("# Local-alignment oracle (+2 / -3 / -3) on synth.workload_local_pair().\n")
        f.write(f"# Written by tests/golden/make_workload_goldens.py ({dt:.1f} s on one core).\n")
        f.write("# fields: M|N|score|a_s|b_s|a_e|b_e|node path length|sha256 of the int32 (K, 2) node path bytes\n")
        f.write(f"{len(X)}|{len(Y)}|{s}|{se[0]}|{se[1]}|{se[2]}|{se[3]}|{len(p)}|{path_sha256(p)}\n")


if __name__ == "__main__":
    main()
