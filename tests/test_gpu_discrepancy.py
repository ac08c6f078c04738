"""The alignment discrepancy of two warping paths (Section 4.3) through the C ABI,
element by element against the oracle's definition."""
import numpy as np
import pytest
import torch

import oracle
import paper_2008_02734_b300 as dtw
from paper_2008_02734_b300 import synth
from tests.test_oracle import random_warping_path

pytestmark = pytest.mark.gpu


def _check(P1, P2, M, N, device):
    r, c = oracle.path_discrepancy(P1, P2)
    a = torch.from_numpy(P1.astype(np.int32))
    b = torch.from_numpy(P2.astype(np.int32))
    if device == "cuda":
        a, b = a.cuda(), b.cuda()
    err, mx = dtw.path_discrepancy(a, b, M, N)
    e = err.cpu().numpy()
    assert e.shape == (2, len(P1))
    assert (e[0] == r).all() and (e[1] == c).all()
    assert mx == max(int(r.max()), int(c.max()))


@pytest.mark.parametrize("M,N", [(1, 1), (1, 9), (9, 1), (2, 2), (17, 5), (40, 63), (300, 257), (1000, 1300)])
@pytest.mark.parametrize("device", ["cuda", "cpu"])
def test_random_paths(M, N, device):
    rng = np.random.default_rng(M * 1000 + N)
    P1, P2 = random_warping_path(rng, M, N), random_warping_path(rng, M, N)
    _check(P1, P2, M, N, device)
    _check(P1, P1, M, N, device)


def test_mixed_host_and_device():
    rng = np.random.default_rng(3)
    M, N = 120, 90
    P1, P2 = random_warping_path(rng, M, N), random_warping_path(rng, M, N)
    r, c = oracle.path_discrepancy(P1, P2)
    err, _ = dtw.path_discrepancy(torch.from_numpy(P1.astype(np.int32)),
                                  torch.from_numpy(P2.astype(np.int32)).cuda(), M, N)
    assert (err[0].numpy() == r).all() and (err[1].numpy() == c).all()


def test_precision_forms_paths_full_size():
    """The exact and BF16 forms' paths of the 60000 x 75000 pair (the paper's use
    of the measure: two alignments of the same pieces)."""
    X, Y = synth.workload_precision()
    M, N = len(X), len(Y)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    p_exact, _ = dtw.align(Xd, Yd)
    p_bf16, _ = dtw.align(Xd, Yd, cost_bf16=True)
    _check(p_exact.cpu().numpy(), p_bf16.cpu().numpy(), M, N, "cuda")
    _check(p_bf16.cpu().numpy(), p_exact.cpu().numpy(), M, N, "cuda")


def _bad(P, M, N):
    return torch.tensor(P, dtype=torch.int32)


@pytest.mark.parametrize("P1", [
    [[0, 0], [1, 1], [1, 3], [2, 3]],   # a step of two columns
    [[0, 0], [1, 1], [0, 2], [2, 3]],   # a step back
    [[0, 1], [1, 1], [2, 2], [2, 3]],   # wrong start
    [[0, 0], [1, 1], [2, 2], [2, 2]],   # repeated cell, wrong end
    [[0, 0], [1, 1], [5, 2], [2, 3]],   # out of range
])
def test_invalid_path_is_rejected(P1):
    good = torch.tensor([[0, 0], [0, 1], [1, 2], [2, 3]], dtype=torch.int32).cuda()
    with pytest.raises(dtw.DTWError) as ei:
        dtw.path_discrepancy(_bad(P1, 3, 4).cuda(), good, 3, 4)
    assert ei.value.status == -1
    with pytest.raises(dtw.DTWError):
        dtw.path_discrepancy(good, _bad(P1, 3, 4).cuda(), 3, 4)


def test_bad_sizes():
    good = torch.tensor([[0, 0], [0, 1], [1, 2], [2, 3]], dtype=torch.int32).cuda()
    with pytest.raises(dtw.DTWError):
        dtw.path_discrepancy(good[:2], good, 3, 4)   # K below max(M, N)
    with pytest.raises(dtw.DTWError):
        dtw.path_discrepancy(good, good, 0, 4)
