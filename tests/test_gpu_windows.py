"""Several split rows per box and level (DTW_OPT_SPLIT_WINDOWS).

Lemma 1 needs only a set of cells that every warping path crosses, and any full
row is one; Lemma 2 then puts the minimisers of F + B - C on each such row on
optimal paths.  A box's two sweeps may therefore end on several windows of split
rows, each fixing a cell, and the box splits into the pieces between them.  The
integer and edit results must stay the oracle's canonical path bit for bit for
every window count (1 is the paper's single middle split); float results within
the float tolerance.  The same cases run with the split fused into the sweep
kernel and as its own launch, with the graph level loop and the host loop.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2008_02734_b300 as dtw
from paper_2008_02734_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6
WINDOWS = [1, 3, 7, 15]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(autouse=True)
def _defaults(cuda_device):
    yield
    dtw.set_option(dtw.OPT_SPLIT_WINDOWS, 7)
    dtw.set_option(dtw.OPT_BASE_AREA, 16384)
    dtw.set_option(dtw.OPT_SWEEP_VARIANT, 0)
    dtw.set_option(dtw.OPT_FUSED_SPLIT, 1)
    dtw.set_option(dtw.OPT_GRAPH, 1)


def _int_exact(X, Y):
    path, cost = dtw.align(_cuda(X), _cuda(Y))
    p_ref, c_ref = oracle.dtw(X, Y)
    assert cost == c_ref
    assert np.array_equal(path.cpu().numpy(), p_ref)


@pytest.mark.parametrize("windows", WINDOWS)
@pytest.mark.parametrize("M,N,base_area", [(129, 257, 4), (500, 433, 64), (1000, 1200, 64), (3000, 2500, 16384),
                                           (5000, 700, 1024), (300, 9000, 4096)])
def test_int_windows_exact(windows, M, N, base_area):
    dtw.set_option(dtw.OPT_SPLIT_WINDOWS, windows)
    dtw.set_option(dtw.OPT_BASE_AREA, base_area)
    X, Y = synth.int_pair(M * 3 + N + windows, M, N)
    _int_exact(X, Y)


@pytest.mark.parametrize("windows", [3, 7, 15])
@pytest.mark.parametrize("alphabet", [2, 3])
def test_int_windows_ties(windows, alphabet):
    """Small alphabets: most windows have no unique minimiser (their pivots are
    left out, or the box is re-swept with split tags); the canonical path stays."""
    rng = np.random.default_rng(17 * alphabet + windows)
    X = rng.integers(0, alphabet, 2500).astype(np.int32)
    Y = rng.integers(0, alphabet, 2100).astype(np.int32)
    dtw.set_option(dtw.OPT_SPLIT_WINDOWS, windows)
    dtw.set_option(dtw.OPT_BASE_AREA, 256)
    _int_exact(X, Y)


def test_int_windows_constant_series():
    X = np.full(3000, 3, np.int32)
    Y = np.full(2200, 1, np.int32)
    dtw.set_option(dtw.OPT_SPLIT_WINDOWS, 7)
    _int_exact(X, Y)
    assert dtw.get_stats()["retagged_boxes"] > 0


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("fused", [0, 2])
@pytest.mark.parametrize("graph", [0, 1])
def test_int_windows_variants_paths(variant, fused, graph):
    dtw.set_option(dtw.OPT_SPLIT_WINDOWS, 7)
    dtw.set_option(dtw.OPT_SWEEP_VARIANT, variant)
    dtw.set_option(dtw.OPT_FUSED_SPLIT, fused)
    dtw.set_option(dtw.OPT_GRAPH, graph)
    X, Y = synth.int_pair(99 + variant, 6000, 7100)
    _int_exact(X, Y)


def test_int_windows_full_pair_levels_and_work():
    """The 20000 x 24000 integer pair: bit-exact, fewer levels than with one
    split row, and the paper's work bound 2MN + (M+N) log2(M+N) still holds."""
    X, Y = synth.workload_int_pair()
    M, N = len(X), len(Y)
    p_ref, c_ref = oracle.dtw(X, Y)
    levels = {}
    for w in (1, 7):
        dtw.set_option(dtw.OPT_SPLIT_WINDOWS, w)
        path, cost = dtw.align(_cuda(X), _cuda(Y))
        assert cost == c_ref
        assert np.array_equal(path.cpu().numpy(), p_ref)
        st = dtw.get_stats()
        levels[w] = st["levels"]
        work = st["sweep_cells"] + st["base_cells"]
        assert work <= 2 * M * N + (M + N) * math.log2(M + N)
    assert levels[7] < levels[1]


@pytest.mark.parametrize("windows", [1, 7, 15])
@pytest.mark.parametrize("M,N,d", [(300, 257, 12), (2000, 2500, 12), (700, 650, 64), (1500, 1800, 5)])
@pytest.mark.parametrize("fused", [0, 1])
def test_float_windows(windows, M, N, d, fused):
    dtw.set_option(dtw.OPT_SPLIT_WINDOWS, windows)
    dtw.set_option(dtw.OPT_FUSED_SPLIT, fused)
    if d == 12:
        X, Y = synth.chroma_pair(M + N, M, N)
    elif d == 64:
        X, Y = synth.mfcc_pair(M + N, M, N)
    else:
        rng = np.random.default_rng(M)
        X = rng.standard_normal((M, d)).astype(np.float32)
        Y = rng.standard_normal((N, d)).astype(np.float32)
    path, cost = dtw.align(_cuda(X), _cuda(Y))
    c_ref = oracle.dtw(X, Y)[1]
    p = path.cpu().numpy()
    assert tuple(p[0]) == (0, 0) and tuple(p[-1]) == (M - 1, N - 1)
    assert cost == pytest.approx(c_ref, rel=REL_TOL)
    assert oracle.path_cost(X, Y, p) == pytest.approx(c_ref, rel=REL_TOL)


@pytest.mark.parametrize("form", ["dp_f32", "cost_bf16"])
def test_reduced_forms_windows(form):
    """The compensated FP32 DP and the BF16 cost form: the same result with one
    split row and with seven windows (both against the oracle's optimum)."""
    X, Y = synth.mfcc_pair(5, 1500, 1700)
    kw = {form: True}
    c_ref = oracle.dtw(X, Y)[1]
    res = {}
    for w in (1, 7):
        dtw.set_option(dtw.OPT_SPLIT_WINDOWS, w)
        path, cost = dtw.align(_cuda(X), _cuda(Y), **kw)
        p = path.cpu().numpy()
        assert tuple(p[0]) == (0, 0) and tuple(p[-1]) == (len(X) - 1, len(Y) - 1)
        tol = 1e-6 if form == "dp_f32" else 5e-3
        assert cost == pytest.approx(c_ref, rel=tol)
        res[w] = cost
    assert res[7] == pytest.approx(res[1], rel=1e-6)


def test_batch_windows_exact():
    """Uneven integer pairs in one batch, seven windows: every pair bit-exact."""
    rng = np.random.default_rng(5)
    Xs, Ys = [], []
    for k in range(24):
        M, N = int(rng.integers(50, 6000)), int(rng.integers(50, 6000))
        X, Y = synth.int_pair(500 + k, M, N)
        Xs.append(X)
        Ys.append(Y)
    dtw.set_option(dtw.OPT_SPLIT_WINDOWS, 7)
    out = dtw.align_batch([_cuda(x) for x in Xs], [_cuda(y) for y in Ys])
    for (path, cost), X, Y in zip(out, Xs, Ys):
        p_ref, c_ref = oracle.dtw(X, Y)
        assert cost == c_ref
        assert np.array_equal(path.cpu().numpy(), p_ref)


@pytest.mark.parametrize("windows", [1, 7])
def test_edit_windows_exact(windows):
    dtw.set_option(dtw.OPT_SPLIT_WINDOWS, windows)
    X, Y = synth.edit_pair(11, 6000)
    path, cost = dtw.edit_align(_cuda(X), _cuda(Y), sub=2, gap=3)
    p_ref, c_ref = oracle.edit(X, Y, sub=2, gap=3)
    assert cost == c_ref
    assert np.array_equal(path.cpu().numpy(), p_ref)

