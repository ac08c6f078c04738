"""Edit distance (Section 5's generalisation) through the same recursion and the
C ABI, against the edit-distance oracle: cost and node path bit for bit (the
canonical DIAG > UP > LEFT path) on every case."""
import hashlib
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2008_02734_b300 as dtw
from paper_2008_02734_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN_EDIT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "edit_20000.txt")


@pytest.fixture(autouse=True)
def _defaults(cuda_device):
    yield
    dtw.set_option(dtw.OPT_BASE_AREA, 16384)
    dtw.set_option(dtw.OPT_EDIT_SUB, 1)
    dtw.set_option(dtw.OPT_EDIT_GAP, 1)


def check_edit(X, Y, sub=1, gap=1, device="cuda"):
    p_ref, c_ref = oracle.edit(X, Y, sub, gap)
    a, b = torch.from_numpy(np.asarray(X, np.int32)), torch.from_numpy(np.asarray(Y, np.int32))
    if device == "cuda":
        a, b = a.cuda(), b.cuda()
    path, cost = dtw.edit_align(a, b, sub=sub, gap=gap)
    assert cost == c_ref
    assert np.array_equal(path.cpu().numpy(), p_ref)
    return path


@pytest.mark.parametrize("M,N", [(1, 1), (1, 7), (7, 1), (2, 3), (17, 9), (64, 64), (130, 257), (1000, 1300),
                                 (3000, 2100)])
@pytest.mark.parametrize("base_area", [64, 16384])
def test_random_pairs(M, N, base_area):
    dtw.set_option(dtw.OPT_BASE_AREA, base_area)
    rng = np.random.default_rng(M * 31 + N)
    X = rng.integers(0, 4, M).astype(np.int32)
    Y = rng.integers(0, 4, N).astype(np.int32)
    check_edit(X, Y)


@pytest.mark.parametrize("sub,gap", [(1, 1), (2, 1), (3, 2), (1, 3), (0, 1), (5, 0)])
def test_weights(sub, gap):
    dtw.set_option(dtw.OPT_BASE_AREA, 64)
    X, Y = synth.edit_pair(sub * 10 + gap, 700, rate=0.2)
    check_edit(X, Y, sub, gap)


@pytest.mark.parametrize("alphabet", [1, 2, 3])
def test_tie_heavy(alphabet):
    """Small alphabets (and a single symbol) make most split rows tie."""
    dtw.set_option(dtw.OPT_BASE_AREA, 64)
    rng = np.random.default_rng(alphabet)
    for M, N in ((300, 410), (513, 97), (64, 1000)):
        X = rng.integers(0, alphabet, M).astype(np.int32)
        Y = rng.integers(0, alphabet, N).astype(np.int32)
        check_edit(X, Y)


def test_mutated_copy_and_host_buffers():
    X, Y = synth.edit_pair(5, 4000)
    check_edit(X, Y, device="cuda")
    check_edit(X, Y, device="cpu")


def test_cost_only_and_batch():
    pairs = [synth.edit_pair(40 + k, 200 + 350 * k) for k in range(6)]
    Xs = [torch.from_numpy(x).cuda() for x, _ in pairs]
    Ys = [torch.from_numpy(y).cuda() for _, y in pairs]
    res = dtw.edit_align_batch(Xs, Ys, sub=2, gap=1)
    for (x, y), (p, c) in zip(pairs, res):
        p_ref, c_ref = oracle.edit(x, y, 2, 1)
        assert c == c_ref
        assert np.array_equal(p.cpu().numpy(), p_ref)
        assert dtw.edit_distance(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), sub=2, gap=1) == c_ref


def test_larger_pair():
    """10000 symbols against a 10%-mutated copy (about 1.2e8 nodes)."""
    X, Y = synth.edit_pair(6, 10000)
    check_edit(X, Y)


def test_full_size_against_stored_oracle():
    """The 20000-symbol workload (unit costs): cost and canonical node path equal
    the edit oracle's, stored by tests/golden/make_workload_goldens.py (the path
    by its length and SHA-256); the one-sweep cost agrees."""
    with open(GOLDEN_EDIT) as f:
        row = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")][-1].split("|")
    M, N, c_ref, K_ref = (int(v) for v in row[:4])
    X, Y = synth.workload_edit_pair()
    assert (len(X), len(Y)) == (M, N)
    path, cost = dtw.edit_align(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    p = path.cpu().numpy()
    assert cost == c_ref
    assert len(p) == K_ref
    assert hashlib.sha256(np.ascontiguousarray(p, dtype="<i4").tobytes()).hexdigest() == row[4]
    assert oracle.edit_path_cost(X, Y, p) == cost
    assert dtw.edit_distance(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()) == cost


def test_overflow_guard_and_bad_input():
    X, Y = synth.edit_pair(7, 1000)
    with pytest.raises(dtw.DTWError) as ei:
        dtw.edit_align(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), sub=1 << 20, gap=1 << 20)
    assert ei.value.status == -5
    with pytest.raises(TypeError):
        dtw.edit_align(torch.zeros(5).cuda(), torch.zeros(6).cuda())
