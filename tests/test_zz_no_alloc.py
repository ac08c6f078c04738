"""dtw_cost_noalloc, the cost entry point that allocates no device memory.

It is meant for callers that cannot call cudaMalloc (device memory reserved up
front by the host application, or work that must not stall on an allocation).
Its scratch is a fixed array inside the library, shared by every call, so these
tests check that back-to-back calls of different sizes give the same D* as
dtw_cost, and that oversized or host inputs are refused.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2008_02734_b300 as dtw
from paper_2008_02734_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


def _noalloc(Xd, Yd):
    """Calls the entry point through the C ABI on the current torch stream."""
    lib = dtw.lib
    M = Xd.shape[0]
    N = Yd.shape[0]
    d = 1 if Xd.dim() == 1 else Xd.shape[1]
    kind = dtw.ABS_I32 if Xd.dtype == torch.int32 else dtw.EUCLID_F32
    c = ctypes.c_double()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dtw_cost_noalloc(ctypes.c_void_p(Xd.data_ptr()), M, ctypes.c_void_p(Yd.data_ptr()), N, d, kind,
                              ctypes.byref(c), st)
    return rc, c.value


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_cost_twice_int(cuda_device):
    # a large call, then a smaller one: the second must not see the first's state
    for seed, (M, N) in enumerate([(6000, 7000), (900, 1300), (6000, 7000)]):
        X, Y = synth.int_pair(70 + seed, M, N)
        Xd, Yd = _cuda(X), _cuda(Y)
        rc, c = _noalloc(Xd, Yd)
        assert rc == dtw.OK
        assert c == dtw.cost(Xd, Yd)


def test_noalloc_matches_cost_twice_float(cuda_device):
    for seed, (M, N) in enumerate([(1200, 1000), (300, 350)]):
        X, Y = synth.chroma_pair(80 + seed, M, N)
        Xd, Yd = _cuda(X), _cuda(Y)
        rc, c = _noalloc(Xd, Yd)
        assert rc == dtw.OK
        assert c == pytest.approx(dtw.cost(Xd, Yd), rel=REL_TOL)


def test_noalloc_rejects_oversize_and_host_inputs(cuda_device):
    lib = dtw.lib
    big = 262144  # DTW_NOALLOC_MAX_SHORT in include/dtw_b300.h
    X = torch.zeros(big + 1, dtype=torch.int32, device="cuda")
    c = ctypes.c_double()
    rc = lib.dtw_cost_noalloc(ctypes.c_void_p(X.data_ptr()), big + 1, ctypes.c_void_p(X.data_ptr()), big + 1, 1,
                              dtw.ABS_I32, ctypes.byref(c), None)
    assert rc == dtw.ENOMEM
    Xh = np.zeros(10, np.int32)
    rc = lib.dtw_cost_noalloc(Xh.ctypes.data, 10, Xh.ctypes.data, 10, 1, dtw.ABS_I32, ctypes.byref(c), None)
    assert rc == dtw.EINVAL
    # still usable afterwards
    Xs, Ys = synth.int_pair(90, 500, 600)
    Xd, Yd = _cuda(Xs), _cuda(Ys)
    rc, v = _noalloc(Xd, Yd)
    assert rc == dtw.OK and v == dtw.cost(Xd, Yd)
