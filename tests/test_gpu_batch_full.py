"""The full uneven batch (256 pairs, M and N in [1000, 20000]) through
dtw_align_batch, every pair against the oracle's stored result
(tests/golden/make_workload_goldens.py calls only oracle/ and the generators).

Chroma-like d=12 pairs (FP32 frame cost): every cost within 1e-6 relative of
oracle 1's FP64 optimum, in both DP forms (FP64 and compensated FP32 pairs), and
every path a warping path whose FP64 re-scoring lies within the same tolerance
(float ties may pick another optimal path, Section 3.2).  Integer pairs: cost and
canonical path bit for bit (the path by its length and SHA-256).
"""
import hashlib
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2008_02734_b300 as dtw
from paper_2008_02734_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip().split("|") for ln in f if ln.strip() and not ln.startswith("#")]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(autouse=True)
def _dev(cuda_device):
    yield


@pytest.mark.parametrize("dp_f32", [False, True])
def test_chroma_batch_256_against_stored_oracle(dp_f32):
    rows = _rows("batch_chroma_256.txt")
    pairs = synth.workload_batch()
    assert len(rows) == len(pairs) == 256
    res = dtw.align_batch([_cuda(x) for x, _ in pairs], [_cuda(y) for _, y in pairs], dp_f32=dp_f32)
    for (X, Y), row, (path, cost) in zip(pairs, rows, res):
        k, M, N, c_ref = int(row[0]), int(row[1]), int(row[2]), float(row[3])
        assert (len(X), len(Y)) == (M, N), k
        p = path.cpu().numpy()
        assert tuple(p[0]) == (0, 0) and tuple(p[-1]) == (M - 1, N - 1), k
        st = np.diff(p, axis=0)
        assert ((st == [0, 1]).all(1) | (st == [1, 0]).all(1) | (st == [1, 1]).all(1)).all(), k
        assert cost == pytest.approx(c_ref, rel=REL_TOL), k
        assert oracle.path_cost(X, Y, p) == pytest.approx(c_ref, rel=REL_TOL), k


def test_int_batch_256_bit_exact_against_stored_oracle():
    rows = _rows("batch_int_256.txt")
    pairs = synth.workload_batch_int()
    assert len(rows) == len(pairs) == 256
    res = dtw.align_batch([_cuda(x) for x, _ in pairs], [_cuda(y) for _, y in pairs])
    for (X, Y), row, (path, cost) in zip(pairs, rows, res):
        k, M, N, c_ref, K_ref = (int(v) for v in row[:5])
        assert (len(X), len(Y)) == (M, N), k
        p = path.cpu().numpy()
        assert cost == c_ref, k
        assert len(p) == K_ref, k
        assert hashlib.sha256(np.ascontiguousarray(p, dtype="<i4").tobytes()).hexdigest() == row[5], k
