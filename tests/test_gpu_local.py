"""Local alignment (Smith-Waterman, named in Section 5) through the C ABI in
linear memory, against the local-alignment oracle: score, start and end nodes
and the node path, bit for bit."""
import hashlib
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2008_02734_b300 as dtw
from paper_2008_02734_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN_LOCAL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "local_20000x24000.txt")


@pytest.fixture(autouse=True)
def _defaults(cuda_device):
    yield
    dtw.set_option(dtw.OPT_BASE_AREA, 16384)


def check_local(X, Y, match=2, mismatch=1, gap=1, device="cuda"):
    p_ref, s_ref, se_ref = oracle.local(X, Y, match, mismatch, gap)
    a, b = torch.from_numpy(np.asarray(X, np.int32)), torch.from_numpy(np.asarray(Y, np.int32))
    if device == "cuda":
        a, b = a.cuda(), b.cuda()
    path, score, se = dtw.local_align(a, b, match=match, mismatch=mismatch, gap=gap)
    assert score == s_ref
    if s_ref == 0:
        assert path.shape[0] == 0
    else:
        assert se == se_ref
        assert np.array_equal(path.cpu().numpy(), p_ref)


@pytest.mark.parametrize("M,N", [(1, 1), (1, 9), (9, 1), (5, 4), (33, 70), (130, 257), (700, 650), (2000, 2600)])
@pytest.mark.parametrize("base_area", [64, 16384])
def test_random_pairs(M, N, base_area):
    dtw.set_option(dtw.OPT_BASE_AREA, base_area)
    rng = np.random.default_rng(M * 37 + N)
    X = rng.integers(0, 4, M).astype(np.int32)
    Y = rng.integers(0, 4, N).astype(np.int32)
    check_local(X, Y)


@pytest.mark.parametrize("match,mismatch,gap", [(2, 1, 1), (1, 1, 1), (3, 2, 2), (5, 4, 1), (1, 3, 2), (2, 0, 0)])
def test_scores(match, mismatch, gap):
    dtw.set_option(dtw.OPT_BASE_AREA, 64)
    X, Y = synth.local_pair(match * 100 + mismatch * 10 + gap, 600, 800, 200)
    check_local(X, Y, match, mismatch, gap)


def test_planted_stretch_and_host_buffers():
    X, Y = synth.local_pair(9, 3000, 3600, 900)
    check_local(X, Y, device="cuda")
    check_local(X, Y, device="cpu")


def test_degenerate():
    check_local(np.array([1, 2, 3], np.int32), np.array([4, 5], np.int32))       # no common symbol
    check_local(np.array([7] * 50, np.int32), np.array([7] * 80, np.int32))       # one symbol: ties everywhere
    X = np.arange(300, dtype=np.int32) % 7
    check_local(X, X.copy())                                                      # identical: the diagonal


def test_full_size_against_stored_oracle():
    """20000 vs 24000 symbols sharing a mutated 5000-symbol stretch, scores
    +2 / -3 / -3: score, start and end nodes and node path equal the oracle's,
    stored by tests/golden/make_workload_goldens.py (the path by its length and
    SHA-256); the path's own score is the local score."""
    with open(GOLDEN_LOCAL) as f:
        row = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")][-1].split("|")
    M, N, s_ref, a_s0, b_s0, a_e0, b_e0, K_ref = (int(v) for v in row[:8])
    X, Y = synth.workload_local_pair()
    assert (len(X), len(Y)) == (M, N)
    path, score, (a_s, b_s, a_e, b_e) = dtw.local_align(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(),
                                                         match=2, mismatch=3, gap=3)
    p = path.cpu().numpy()
    assert score == s_ref
    assert (a_s, b_s, a_e, b_e) == (a_s0, b_s0, a_e0, b_e0)
    assert len(p) == K_ref
    assert hashlib.sha256(np.ascontiguousarray(p, dtype="<i4").tobytes()).hexdigest() == row[8]
    sc = 0
    for (a0, b0), (a1, b1) in zip(p[:-1], p[1:]):
        sc += (2 if X[a1 - 1] == Y[b1 - 1] else -3) if (a1 - a0 == 1 and b1 - b0 == 1) else -3
    assert sc == score
