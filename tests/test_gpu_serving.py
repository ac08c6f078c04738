"""The request engine behind dtw_submit / dtw_poll (continuous batching).

Requests of mixed sizes, kinds and buffer locations go in at different times;
each result must equal what dtw_align returns for the same pair alone (integer
kind: bit for bit; float kind: within the float tolerance), and a request that
arrives while a long one is in flight must be admitted next to it and finish
first instead of queueing behind it.
"""
import time

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


# The BF16 form against its own cost model (the oracle's BF16-form costs under
# oracle 1's DP; the GPU takes norms and dot products in FP32): 2e-4 relative.
BF16_FORM_TOL = 2e-4
# The BF16 form against the exact FP64 optimum, for these short d=64 pairs (1 to
# 1500 frames): 5e-3 relative.  A cell's cost moves by up to
# sqrt(2^-7 |x| |y|) where frames are near-identical, and a short path averages
# few cells (one pair here measured 1.03e-3; the 60000 x 75000 pair, 4.9e-5
# against its stated 1e-3).
BF16_EXACT_TOL = 5e-3


def _alone(X, Y, **form):
    path, cost = dtw.align(_cuda(X), _cuda(Y), **form)
    return path.cpu().numpy(), cost


def test_mixed_stream_matches_alone():
    """Integer, chroma d=12 and MFCC-like d=64 requests (the d=64 ones in the
    exact FP32-cost form and in the BF16 tensor-core form), on host and device
    buffers, submitted in waves while earlier ones run: every result equals the
    same pair aligned alone by dtw_align in the same form (integer: bit for bit;
    float forms: 1e-6 relative); against the FP64 oracle the exact forms lie
    within 1e-6 (cost, and the path re-scored in FP64); the BF16 form lies within
    2e-4 of the oracle's optimum of the BF16-form costs (cost and re-scored path)
    and within 5e-3 of the exact FP64 optimum."""
    rng = np.random.default_rng(7)
    jobs = []
    for k in range(32):
        M = int(rng.integers(1, 3000))
        N = int(rng.integers(1, 3000))
        form = {}
        if k % 4 == 2:
            X, Y = synth.chroma_pair(1000 + k, M, N)
        elif k % 4 == 3:
            X, Y = synth.mfcc_pair(1000 + k, M // 2 + 1, N // 2 + 1)
            form = {"cost_bf16": True} if k % 8 == 7 else {}
        else:
            X, Y = synth.int_pair(1000 + k, M, N)
        on_dev = k % 2 == 0
        jobs.append((X, Y, on_dev, form))
    tickets = []
    for i, (X, Y, on_dev, form) in enumerate(jobs):
        xs, ys = (_cuda(X), _cuda(Y)) if on_dev else (X, Y)
        path_buf = None if on_dev else torch.empty((len(X) + len(Y) - 1, 2), dtype=torch.int32)
        tickets.append(dtw.submit(xs, ys, path_out=path_buf, **form))
        if i % 5 == 4:  # let earlier requests get under way before more arrive
            time.sleep(2e-3)
    for (X, Y, on_dev, form), (t, path, keep) in zip(jobs, tickets):
        rc, K, c = dtw.wait(t)
        assert rc == dtw.OK, dtw.DTWError(rc, "serve")
        p = path[:K].cpu().numpy()
        p_ref, c_ref = _alone(X, Y, **form)
        if X.dtype == np.int32:
            assert c == c_ref
            assert np.array_equal(p, p_ref)
            assert c == oracle.dtw(X, Y)[1]
        elif form.get("cost_bf16"):
            assert c == pytest.approx(c_ref, rel=REL_TOL, abs=1e-9)
            C = oracle.bf16_form_costs(X, Y)
            c_form = oracle.dtw_given(C)[1]
            assert c == pytest.approx(c_form, rel=BF16_FORM_TOL, abs=1e-6)
            assert C[p[:, 0], p[:, 1]].sum() == pytest.approx(c_form, rel=BF16_FORM_TOL, abs=1e-6)
            assert c == pytest.approx(oracle.dtw(X, Y)[1], rel=BF16_EXACT_TOL, abs=1e-6)
        else:
            assert c == pytest.approx(c_ref, rel=REL_TOL, abs=1e-9)
            c_opt = oracle.dtw(X, Y)[1]
            assert c == pytest.approx(c_opt, rel=REL_TOL, abs=1e-9)
            assert oracle.path_cost(X, Y, p) == pytest.approx(c_opt, rel=REL_TOL, abs=1e-9)


def test_late_request_admitted_while_long_one_runs():
    """A short request submitted right after a long one of the same group joins
    its levels instead of queueing behind it: it finishes while the long one
    (a 100000 x 120000 integer pair, some ten levels) is still in flight.  Both
    results: the short one equals the oracle's bit for bit, the long one equals
    the pair aligned alone (the full-size oracle would take too long here)."""
    import time
    Xb, Yb = synth.int_pair(1, 100000, 120000)
    Xs, Ys = synth.int_pair(77, 600, 700)
    Xbd, Ybd, Xsd, Ysd = _cuda(Xb), _cuda(Yb), _cuda(Xs), _cuda(Ys)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tb, pb, kb = dtw.submit(Xbd, Ybd)
    ts, ps, ks = dtw.submit(Xsd, Ysd)
    rc, K, c = dtw.wait(ts, interval_s=2e-5)
    t_short = time.perf_counter() - t0
    assert rc == dtw.OK
    # the short request finished while the long one was still being aligned
    st_long = dtw.poll(tb)[0]
    rcb, Kb, cb = dtw.wait(tb, interval_s=2e-5)
    t_long = time.perf_counter() - t0
    print(f"short request {1e3 * t_short:.2f} ms, long request {1e3 * t_long:.2f} ms")
    assert st_long == dtw.PENDING
    p_ref, c_ref = oracle.dtw(Xs, Ys)
    assert c == c_ref and np.array_equal(ps[:K].cpu().numpy(), p_ref)
    assert rcb == dtw.OK
    p_alone, c_alone = _alone(Xb, Yb)
    assert cb == c_alone and np.array_equal(pb[:Kb].cpu().numpy(), p_alone)


def test_groups_overlap_short_d64_during_long_d12():
    """The d=12 and d=64 groups have their own engines (threads and streams):
    a short d=64 request submitted right after a long d=12 one is not served
    level by level in turn with it.  It finishes while the long one is still in
    flight, within half the long one's latency (alternating the groups' levels,
    it would wait for a level of the long pair before each of its own), and both
    results equal the pairs aligned alone."""
    import time
    # the long request long enough (about 25 ms alone) that one of its levels
    # outlasts the short request many times over
    Xl, Yl = synth.chroma_pair(501, 30000, 36000)
    Xs, Ys = synth.mfcc_pair(502, 700, 800)
    dl, ds = (_cuda(Xl), _cuda(Yl)), (_cuda(Xs), _cuda(Ys))
    # warm both engines up (arena creation is not part of the measurement)
    for X, Y in (dl, ds):
        assert dtw.wait(dtw.submit(X, Y)[0])[0] == dtw.OK
    t0 = time.perf_counter()
    tl, pl, kl = dtw.submit(*dl)
    ts, ps, ks = dtw.submit(*ds)
    rc, Ks, cs = dtw.wait(ts, interval_s=2e-5)
    t_short = time.perf_counter() - t0
    assert rc == dtw.OK
    long_pending = dtw.poll(tl)[0] == dtw.PENDING
    rc, Kl, cl = dtw.wait(tl, interval_s=2e-5)
    t_long = time.perf_counter() - t0
    assert rc == dtw.OK
    print(f"short d=64 request {1e3 * t_short:.2f} ms, long d=12 request {1e3 * t_long:.2f} ms")
    assert long_pending
    assert t_short < 0.5 * t_long
    ref_s = _alone(Xs, Ys)
    assert cs == pytest.approx(ref_s[1], rel=REL_TOL)
    assert oracle.path_cost(Xs, Ys, ps[:Ks].cpu().numpy()) == pytest.approx(ref_s[1], rel=REL_TOL)
    ref_l = _alone(Xl, Yl)
    assert cl == pytest.approx(ref_l[1], rel=REL_TOL)


def test_overflowing_request_fails_alone():
    bad = dtw.submit(_cuda(np.array([0, 2 ** 30], np.int32)), _cuda(np.array([-2 ** 30, 5, 7], np.int32)))
    X, Y = synth.int_pair(78, 500, 400)
    good = dtw.submit(_cuda(X), _cuda(Y))
    assert dtw.wait(bad[0])[0] == dtw.EOVERFLOW
    rc, K, c = dtw.wait(good[0])
    assert rc == dtw.OK and c == oracle.dtw(X, Y)[1]


def test_unknown_ticket():
    assert dtw.poll(10 ** 12)[0] == dtw.EINVAL
