"""dtw_cost_noalloc, the cost entry point that allocates no device memory.

It is meant for callers that cannot call cudaMalloc (device memory reserved up
front by the host application, or work that must not stall on an allocation).
Its scratch is a fixed array inside the library, shared by every call, so these
tests check back-to-back calls of different sizes and kinds against the CPU
oracle (integer kind: D* bit for bit; float kinds: within 1e-6 relative) and
against dtw_cost, pairs with either side the longer one, the short side at the
array's limit (against closed forms), calls on another stream, the restart of
the boundary-word epochs near the 32-bit limit, and the refusals (oversized,
host or misaligned inputs).

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2008_02734_b300 as dtw
from paper_2008_02734_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6
MAX_SHORT = 262144  # DTW_NOALLOC_MAX_SHORT in include/dtw_b300.h
MAX_LONG = 4194304  # DTW_NOALLOC_MAX_LONG


def _noalloc_raw(xp, M, yp, N, d, kind, stream=None):
    c = ctypes.c_double()
    st = ctypes.c_void_p(stream)
    rc = dtw.lib.dtw_cost_noalloc(ctypes.c_void_p(xp), M, ctypes.c_void_p(yp), N, d, kind, ctypes.byref(c), st)
    return rc, c.value


def _noalloc(Xd, Yd, stream=None):
    """Calls the entry point through the C ABI (on the current torch stream
    unless a stream is given)."""
    d = 1 if Xd.dim() == 1 else Xd.shape[1]
    kind = dtw.ABS_I32 if Xd.dtype == torch.int32 else dtw.EUCLID_F32
    s = (stream or torch.cuda.current_stream()).cuda_stream
    return _noalloc_raw(Xd.data_ptr(), Xd.shape[0], Yd.data_ptr(), Yd.shape[0], d, kind, s)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_int_against_oracle_back_to_back(cuda_device):
    # a large call, then a smaller one, then a transposed one: each must equal the
    # oracle's D* bit for bit and not see the previous call's state
    for seed, (M, N) in enumerate([(6000, 7000), (900, 1300), (7000, 6000), (1, 500), (500, 1)]):
        X, Y = synth.int_pair(70 + seed, M, N)
        Xd, Yd = _cuda(X), _cuda(Y)
        rc, c = _noalloc(Xd, Yd)
        assert rc == dtw.OK
        assert c == oracle.dtw(X, Y)[1]
        assert c == dtw.cost(Xd, Yd)


@pytest.mark.parametrize("d,shapes", [(12, [(1200, 1000), (300, 350)]), (64, [(700, 500), (400, 650)]),
                                      (5, [(900, 700), (333, 444)])])
def test_noalloc_float_against_oracle(cuda_device, d, shapes):
    for seed, (M, N) in enumerate(shapes):
        if d == 12:
            X, Y = synth.chroma_pair(80 + seed, M, N)
        else:
            X, Y = synth.mfcc_pair(80 + seed, M, N, d=d)
        Xd, Yd = _cuda(X), _cuda(Y)
        rc, c = _noalloc(Xd, Yd)
        assert rc == dtw.OK
        assert c == pytest.approx(oracle.dtw(X, Y)[1], rel=REL_TOL)
        assert c == pytest.approx(dtw.cost(Xd, Yd), rel=REL_TOL)


def _stutter(rng, Y, M):
    """X = Y with M - len(Y) of its frames repeated once (in place): a warping
    path maps every copy onto its original, so D*(X, Y) = 0."""
    N = len(Y)
    reps = np.zeros(N, dtype=np.int64)
    reps[rng.choice(N, M - N, replace=False)] = 1
    return np.repeat(Y, 1 + reps, axis=0)


def test_noalloc_short_side_at_limit_closed_forms(cuda_device):
    """The short side at the fixed array's limit, the long side the rows (M > N):
    a stuttered copy has D* = 0 (integer and chroma frames), constant series
    a and b have D* = |a - b| max(M, N)."""
    rng = np.random.default_rng(5)
    N, M = MAX_SHORT, 300000
    Y = rng.integers(0, 256, N).astype(np.int32)
    X = _stutter(rng, Y, M)
    assert len(X) == M
    rc, c = _noalloc(_cuda(X), _cuda(Y))
    assert rc == dtw.OK and c == 0.0
    rc, c = _noalloc(_cuda(Y), _cuda(X))  # transposed: the short side on X
    assert rc == dtw.OK and c == 0.0
    rc, c = _noalloc(_cuda(np.full(M, 7, np.int32)), _cuda(np.full(N, 3, np.int32)))
    assert rc == dtw.OK and c == 4.0 * M
    Yf = synth.chroma_walk(rng, N)
    Xf = _stutter(rng, Yf, M)
    rc, c = _noalloc(_cuda(Xf), _cuda(Yf))
    assert rc == dtw.OK and c == 0.0


def test_noalloc_on_another_stream(cuda_device):
    X, Y = synth.int_pair(91, 2500, 2200)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Xd, Yd = _cuda(X), _cuda(Y)
        rc, c = _noalloc(Xd, Yd, stream=s)
    s.synchronize()
    assert rc == dtw.OK and c == oracle.dtw(X, Y)[1]


def test_noalloc_epoch_restart_near_32_bits(cuda_device):
    """Start the epochs just below the 32-bit limit (test hook): the call that
    could wrap restarts them at 1 and clears the boundary row; every call still
    gives the oracle's D*."""
    X, Y = synth.int_pair(92, 3000, 3300)
    Xd, Yd = _cuda(X), _cuda(Y)
    c_ref = oracle.dtw(X, Y)[1]
    for start in (2 ** 32 - 200, 2 ** 32 - 1, 2 ** 32 - 200000, 0):
        dtw.set_option(dtw.OPT_NOALLOC_EPOCH, start)
        for _ in range(3):
            rc, c = _noalloc(Xd, Yd)
            assert rc == dtw.OK and c == c_ref, start


def test_noalloc_rejects_oversize_host_and_misaligned_inputs(cuda_device):
    small = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = small.data_ptr()
    # sizes past the fixed array are refused before any memory is read
    assert _noalloc_raw(p, MAX_SHORT + 1, p, MAX_SHORT + 1, 1, dtw.ABS_I32)[0] == dtw.ENOMEM
    assert _noalloc_raw(p, MAX_LONG + 1, p, 10, 1, dtw.ABS_I32)[0] == dtw.ENOMEM
    assert _noalloc_raw(p, 10, p, MAX_LONG + 1, 1, dtw.ABS_I32)[0] == dtw.ENOMEM
    Xh = np.zeros(10, np.int32)
    assert _noalloc_raw(Xh.ctypes.data, 10, Xh.ctypes.data, 10, 1, dtw.ABS_I32)[0] == dtw.EINVAL
    # d = 12 frames are read in 16-byte pieces: a 4-byte offset is refused
    F = torch.zeros((20, 12), dtype=torch.float32, device="cuda")
    assert _noalloc_raw(F.data_ptr() + 4, 10, F.data_ptr(), 10, 12, dtw.EUCLID_F32)[0] == dtw.EINVAL
    # bad kinds and dimensions
    assert _noalloc_raw(p, 4, p, 4, 2, dtw.ABS_I32)[0] == dtw.EINVAL
    assert _noalloc_raw(p, 4, p, 4, 1, 7)[0] == dtw.EINVAL
    # still usable afterwards
    Xs, Ys = synth.int_pair(90, 500, 600)
    rc, v = _noalloc(_cuda(Xs), _cuda(Ys))
    assert rc == dtw.OK and v == oracle.dtw(Xs, Ys)[1]
