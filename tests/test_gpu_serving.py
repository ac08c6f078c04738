"""The request engine behind dtw_submit / dtw_poll (continuous batching).

Requests of mixed sizes, kinds and buffer locations go in at different times;
each result must equal what dtw_align returns for the same pair alone (integer
kind: bit for bit; float kind: within the float tolerance), and a request that
arrives while a long one is in flight must be admitted next to it and finish
first instead of queueing behind it.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2008_02734_b300 as dtw
from paper_2008_02734_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(autouse=True)
def _dev(cuda_device):
    yield


def _alone(X, Y):
    path, cost = dtw.align(_cuda(X), _cuda(Y))
    return path.cpu().numpy(), cost


def test_mixed_stream_matches_alone():
    rng = np.random.default_rng(7)
    jobs = []
    for k in range(24):
        M = int(rng.integers(1, 3000))
        N = int(rng.integers(1, 3000))
        if k % 3 == 2:
            X, Y = synth.chroma_pair(1000 + k, M, N)
        else:
            X, Y = synth.int_pair(1000 + k, M, N)
        on_dev = k % 2 == 0
        jobs.append((X, Y, on_dev))
    tickets = []
    for i, (X, Y, on_dev) in enumerate(jobs):
        xs, ys = (_cuda(X), _cuda(Y)) if on_dev else (X, Y)
        path_buf = None if on_dev else torch.empty((len(X) + len(Y) - 1, 2), dtype=torch.int32)
        tickets.append(dtw.submit(xs, ys, path_out=path_buf))
        if i % 5 == 4:  # let earlier requests get under way before more arrive
            dtw.poll(tickets[0][0])
    for (X, Y, on_dev), (t, path, keep) in zip(jobs, tickets):
        rc, K, c = dtw.wait(t)
        assert rc == dtw.OK, dtw.DTWError(rc, "serve")
        p = path[:K].cpu().numpy()
        p_ref, c_ref = _alone(X, Y)
        if X.dtype == np.int32:
            assert c == c_ref
            assert np.array_equal(p, p_ref)
            assert c == oracle.dtw(X, Y)[1]
        else:
            assert c == pytest.approx(c_ref, rel=REL_TOL, abs=1e-9)
            assert oracle.path_cost(X, Y, p) == pytest.approx(oracle.dtw(X, Y)[1], rel=REL_TOL, abs=1e-9)


def test_late_request_admitted_while_long_one_runs():
    Xb, Yb = synth.workload_int_pair()
    Xs, Ys = synth.int_pair(77, 600, 700)
    tb, pb, kb = dtw.submit(_cuda(Xb), _cuda(Yb))
    ts, ps, ks = dtw.submit(_cuda(Xs), _cuda(Ys))
    rc, K, c = dtw.wait(ts)
    assert rc == dtw.OK
    # the short request finished while the long one was still being aligned
    assert dtw.poll(tb)[0] == dtw.PENDING
    p_ref, c_ref = oracle.dtw(Xs, Ys)
    assert c == c_ref and np.array_equal(ps[:K].cpu().numpy(), p_ref)
    rc, K, c = dtw.wait(tb)
    assert rc == dtw.OK
    assert c == oracle.dtw(Xb, Yb)[1]


def test_overflowing_request_fails_alone():
    bad = dtw.submit(_cuda(np.array([0, 2 ** 30], np.int32)), _cuda(np.array([-2 ** 30, 5, 7], np.int32)))
    X, Y = synth.int_pair(78, 500, 400)
    good = dtw.submit(_cuda(X), _cuda(Y))
    assert dtw.wait(bad[0])[0] == dtw.EOVERFLOW
    rc, K, c = dtw.wait(good[0])
    assert rc == dtw.OK and c == oracle.dtw(X, Y)[1]


def test_unknown_ticket():
    assert dtw.poll(10 ** 12)[0] == dtw.EINVAL
