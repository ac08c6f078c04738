"""Pins of the CPU oracle to things other than itself (runs without a GPU).

* brute-force enumeration of every warping path (M, N <= 7), whose path count is
  checked against the Delannoy closed form;
* hand-derived examples in tests/golden/handworked.txt;
* closed forms (identical series, constant series, a single row);
* invariants: endpoints, step set, the path's cost equals D*, reversal and
  transposition invariance of D*, Lemma 2's split identity on every row, and the
  work bound of Section 3.2 for oracle 2;
* the alignment discrepancy of Section 4.3 against hand-worked cases
  (tests/golden/discrepancy.txt), against the run-extent closed form on random
  monotone paths, and its zero and symmetry properties.
"""
import math
import os

import numpy as np
import pytest

import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "handworked.txt")


def _rows(s, kind):
    frames = [r.split(",") for r in s.split(";")]
    if kind == "int":
        return np.array([int(f[0]) for f in frames], dtype=np.int32)
    return np.array([[float(v) for v in f] for f in frames], dtype=np.float32)


def _golden_cases():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, kind, xs, ys, ds, cost, ps = line.split("|")
        X, Y = _rows(xs, kind), _rows(ys, kind)
        D = np.array([[float(v) for v in r.split(",")] for r in ds.split(";")])
        path = np.array([[int(v) for v in c.split(",")] for c in ps.split(";")], dtype=np.int32)
        out.append((name, X, Y, D, float(cost), path))
    return out


def check_path(path, M, N):
    path = np.asarray(path)
    assert tuple(path[0]) == (0, 0)
    assert tuple(path[-1]) == (M - 1, N - 1)
    steps = np.diff(path, axis=0)
    ok = {(0, 1), (1, 0), (1, 1)}
    assert all(tuple(s) in ok for s in steps), "illegal step"
    assert max(M, N) <= len(path) <= M + N - 1


def np_path_cost(X, Y, path):
    """Sum of frame costs along a path, computed with numpy (independent of the oracle)."""
    path = np.asarray(path)
    if X.dtype == np.int32:
        return int(np.abs(X[path[:, 0]].astype(np.int64) - Y[path[:, 1]].astype(np.int64)).sum())
    Xd = X.reshape(len(X), -1).astype(np.float64)
    Yd = Y.reshape(len(Y), -1).astype(np.float64)
    return float(np.linalg.norm(Xd[path[:, 0]] - Yd[path[:, 1]], axis=1).sum())


# ---------------------------------------------------------------- brute force

def test_enumerator_counts_match_delannoy():
    for M in range(1, 8):
        for N in range(1, 8):
            assert len(brute.all_paths(M, N)) == brute.delannoy(M - 1, N - 1)
    assert brute.delannoy(6, 6) == 8989


@pytest.mark.parametrize("alphabet", [2, 3, 5, 256])
def test_int_cost_and_canonical_path_vs_brute_force(alphabet):
    rng = np.random.default_rng(100 + alphabet)
    for _ in range(60):
        M, N = (int(v) for v in rng.integers(1, 8, 2))
        X = rng.integers(0, alphabet, M).astype(np.int32)
        Y = rng.integers(0, alphabet, N).astype(np.int32)
        best, canon, _, _ = brute.solve(X, Y)
        path, cost = oracle.dtw(X, Y)
        assert cost == best
        assert [tuple(c) for c in path] == canon


def test_float_cost_vs_brute_force():
    rng = np.random.default_rng(7)
    for _ in range(60):
        M, N = (int(v) for v in rng.integers(1, 7, 2))
        d = int(rng.integers(1, 4))
        X = rng.standard_normal((M, d)).astype(np.float32)
        Y = rng.standard_normal((N, d)).astype(np.float32)
        best, canon, nopt, _ = brute.solve(X, Y)
        path, cost = oracle.dtw(X, Y)
        # the DP minimum equals the minimum over paths of first-to-last sums, bit for bit
        assert cost == best
        check_path(path, M, N)
        s = 0.0
        C = brute.cost_table(X, Y)
        for (i, j) in path:
            s = s + C[i][j]
        assert s == best
        if nopt == 1:
            assert [tuple(c) for c in path] == canon


def test_acc_matrices_vs_brute_force():
    rng = np.random.default_rng(11)
    for _ in range(8):
        M, N = (int(v) for v in rng.integers(1, 6, 2))
        X = rng.integers(0, 4, M).astype(np.int32)
        Y = rng.integers(0, 4, N).astype(np.int32)
        F = oracle.acc_matrix(X, Y)
        B = oracle.acc_matrix(X, Y, reverse=True)
        for i in range(M):
            for j in range(N):
                assert F[i, j] == brute.prefix_optimum(X, Y, i, j)
                assert B[i, j] == brute.suffix_optimum(X, Y, i, j)


# ---------------------------------------------------------------- hand-worked

@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_handworked(case):
    name, X, Y, D, cost, gpath = case
    path, c = oracle.dtw(X, Y)
    assert c == cost
    assert np.array_equal(path, gpath)
    assert np.array_equal(oracle.acc_matrix(X, Y).astype(np.float64), D)


# ---------------------------------------------------------------- closed forms

def test_identical_series_cost_zero_on_diagonal():
    rng = np.random.default_rng(3)
    for M in (1, 2, 17, 64):
        X = rng.standard_normal((M, 5)).astype(np.float32)
        path, cost = oracle.dtw(X, X.copy())
        assert cost == 0.0
        assert np.array_equal(path, np.stack([np.arange(M)] * 2, 1))
        Xi = rng.integers(-50, 50, M).astype(np.int32)
        path, cost = oracle.dtw(Xi, Xi.copy())
        assert cost == 0 and np.array_equal(path, np.stack([np.arange(M)] * 2, 1))


@pytest.mark.parametrize("M,N", [(3, 9), (9, 3), (5, 5), (1, 7), (7, 1), (40, 53)])
@pytest.mark.parametrize("a,b", [(4, 9), (6, 6)])
def test_constant_series(M, N, a, b):
    X = np.full(M, a, np.int32)
    Y = np.full(N, b, np.int32)
    path, cost = oracle.dtw(X, Y)
    assert cost == abs(a - b) * max(M, N)
    # canonical path: DIAG from the last cell while both indices move, then the
    # remaining run along row 0 (M <= N) or column 0 (M > N)
    if M <= N:
        expect = [(0, j) for j in range(N - M + 1)] + [(k, N - M + k) for k in range(1, M)]
    else:
        expect = [(i, 0) for i in range(M - N + 1)] + [(M - N + k, k) for k in range(1, N)]
    assert [tuple(c) for c in path] == expect


def test_single_row_is_row_sum():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((31, 3)).astype(np.float32)
    X = rng.standard_normal((1, 3)).astype(np.float32)
    path, cost = oracle.dtw(X, Y)
    assert np.array_equal(path, np.stack([np.zeros(31, int), np.arange(31)], 1))
    assert cost == pytest.approx(np.linalg.norm(Y.astype(np.float64) - X[0], axis=1).sum(), rel=1e-14)


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(4))
def test_invariants_medium(seed):
    rng = np.random.default_rng(seed)
    M, N = (int(v) for v in rng.integers(20, 90, 2))
    X = rng.integers(0, 20, M).astype(np.int32)
    Y = rng.integers(0, 20, N).astype(np.int32)
    path, cost = oracle.dtw(X, Y)
    check_path(path, M, N)
    assert np_path_cost(X, Y, path) == cost
    assert oracle.path_cost(X, Y, path) == cost
    # reversal and transposition leave D* unchanged
    assert oracle.dtw(X[::-1].copy(), Y[::-1].copy())[1] == cost
    assert oracle.dtw(Y, X)[1] == cost
    Xf = rng.standard_normal((M, 4)).astype(np.float32)
    Yf = rng.standard_normal((N, 4)).astype(np.float32)
    pf, cf = oracle.dtw(Xf, Yf)
    check_path(pf, M, N)
    assert np_path_cost(Xf, Yf, pf) == pytest.approx(cf, rel=1e-12)
    assert oracle.dtw(Xf[::-1].copy(), Yf[::-1].copy())[1] == pytest.approx(cf, rel=1e-12)
    assert oracle.dtw(Yf, Xf)[1] == pytest.approx(cf, rel=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_split_identity_every_row(seed):
    """Lemma 2: F + B - C is D* on every cell of an optimal path, and its minimum
    over any row is D*."""
    rng = np.random.default_rng(20 + seed)
    M, N = (int(v) for v in rng.integers(10, 50, 2))
    X = rng.integers(0, 8, M).astype(np.int32)
    Y = rng.integers(0, 8, N).astype(np.int32)
    path, cost = oracle.dtw(X, Y)
    F = oracle.acc_matrix(X, Y)
    B = oracle.acc_matrix(X, Y, reverse=True)
    C = np.abs(X[:, None].astype(np.int64) - Y[None, :].astype(np.int64))
    S = F + B - C
    assert (S.min(axis=1) == cost).all()
    assert (S.min(axis=0) == cost).all()
    assert (S[path[:, 0], path[:, 1]] == cost).all()
    assert F[-1, -1] == cost and B[0, 0] == cost


# ---------------------------------------------------------------- oracle 2

@pytest.mark.parametrize("m", [3, 4, 8])
def test_linmdtw_matches_textbook(m):
    rng = np.random.default_rng(30 + m)
    for t in range(40):
        M, N = (int(v) for v in rng.integers(1, 60, 2))
        X = rng.integers(0, 6, M).astype(np.int32)
        Y = rng.integers(0, 6, N).astype(np.int32)
        p1, c1 = oracle.dtw(X, Y)
        p2, c2, cells = oracle.linmdtw(X, Y, m=m)
        check_path(p2, M, N)
        assert c2 == c1
        assert np_path_cost(X, Y, p2) == c1


def test_linmdtw_float_and_brute_force():
    rng = np.random.default_rng(41)
    for _ in range(30):
        M, N = (int(v) for v in rng.integers(3, 7, 2))
        X = rng.standard_normal((M, 2)).astype(np.float32)
        Y = rng.standard_normal((N, 2)).astype(np.float32)
        best = brute.solve(X, Y)[0]
        p2, c2, _ = oracle.linmdtw(X, Y, m=3)
        check_path(p2, M, N)
        assert c2 == pytest.approx(best, rel=1e-12)


def test_linmdtw_work_bound():
    """Section 3.2: at most 2MN + (M+N) log2(M+N) cells, about 2MN in practice."""
    from paper_2008_02734_b300 import synth
    for seed, (M, N) in enumerate([(300, 360), (500, 400), (900, 1100)]):
        X, Y = synth.int_pair(seed, M, N)
        p, c, cells = oracle.linmdtw(X, Y, m=20)
        assert cells <= 2 * M * N + (M + N) * math.log2(M + N)
        assert 1.6 < cells / (M * N) <= 2.1
        assert c == oracle.dtw(X, Y)[1]


DISC_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "discrepancy.txt")


def _pairs(s):
    return np.array([[int(v) for v in c.split(",")] for c in s.split(";")], dtype=np.int64)


def _disc_cases():
    with open(DISC_GOLDEN) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                name, M, N, p1, p2, re, ce = ln.split("|")
                yield name, int(M), int(N), _pairs(p1), _pairs(p2), [int(v) for v in re.split(",")], \
                    [int(v) for v in ce.split(",")]


@pytest.mark.parametrize("case", list(_disc_cases()), ids=lambda c: c[0])
def test_discrepancy_handworked(case):
    name, M, N, P1, P2, re, ce = case
    r, c = oracle.path_discrepancy(P1, P2)
    assert r.tolist() == re and c.tolist() == ce


def random_warping_path(rng, M, N):
    """A seeded random warping path from (0,0) to (M-1,N-1) (test input)."""
    i = j = 0
    out = [(0, 0)]
    while (i, j) != (M - 1, N - 1):
        moves = [m for m in ((1, 1), (1, 0), (0, 1)) if i + m[0] < M and j + m[1] < N]
        di, dj = moves[rng.integers(len(moves))]
        i, j = i + di, j + dj
        out.append((i, j))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("seed", range(6))
def test_discrepancy_closed_form_on_random_paths(seed):
    """A warping path's cells in one row form one run [lo, hi] (steps never go
    back), so the row error of (i, j) is max(0, lo_i - j, j - hi_i); likewise for
    columns.  The oracle compares every cell and must agree."""
    rng = np.random.default_rng(seed)
    M, N = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    P1, P2 = random_warping_path(rng, M, N), random_warping_path(rng, M, N)
    lo = {int(i): int(P2[P2[:, 0] == i, 1].min()) for i in range(M)}
    hi = {int(i): int(P2[P2[:, 0] == i, 1].max()) for i in range(M)}
    clo = {int(j): int(P2[P2[:, 1] == j, 0].min()) for j in range(N)}
    chi = {int(j): int(P2[P2[:, 1] == j, 0].max()) for j in range(N)}
    r, c = oracle.path_discrepancy(P1, P2)
    for t, (i, j) in enumerate(P1):
        assert r[t] == max(0, lo[int(i)] - j, j - hi[int(i)])
        assert c[t] == max(0, clo[int(j)] - i, i - chi[int(j)])


def test_discrepancy_zero_and_symmetry():
    """A path against itself has no error; swapping the roles of rows and
    columns (transposing both paths) swaps row and column errors."""
    rng = np.random.default_rng(7)
    P1, P2 = random_warping_path(rng, 25, 31), random_warping_path(rng, 25, 31)
    r, c = oracle.path_discrepancy(P1, P1)
    assert not r.any() and not c.any()
    r, c = oracle.path_discrepancy(P1, P2)
    rt, ct = oracle.path_discrepancy(P1[:, ::-1], P2[:, ::-1])
    assert (rt == c).all() and (ct == r).all()


# ------------------------------------------ oracle 1 on a given cost matrix

@pytest.mark.parametrize("levels", [2, 3, 1000])
def test_dtw_given_vs_brute_force(levels):
    """Cost and canonical path over explicit matrices; few distinct values make
    many optimal paths, so the tie order DIAG, UP, LEFT is exercised."""
    rng = np.random.default_rng(300 + levels)
    for _ in range(60):
        M, N = (int(v) for v in rng.integers(1, 7, 2))
        C = rng.integers(0, levels, (M, N)).astype(np.float64) * 0.25
        best, canon, _, _ = brute.solve_table(C)
        path, cost = oracle.dtw_given(C)
        assert cost == best
        assert [tuple(c) for c in path] == canon


def test_dtw_given_equals_oracle_on_euclidean_costs():
    """Handing oracle 1's own frame costs in as a matrix changes nothing."""
    X, Y = np.random.default_rng(5).standard_normal((2, 40, 3)).astype(np.float32)
    C = np.array(brute.cost_table(X, Y))
    p1, c1 = oracle.dtw(X, Y)
    p2, c2 = oracle.dtw_given(C)
    assert c1 == c2 and np.array_equal(p1, p2)


# ------------------------------------------ the BF16 tensor-core cost form

def test_bf16_round_ties_to_even_and_matches_torch():
    one = np.float32(1.0)
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even 1
    assert oracle.bf16_round(np.float32(1 + 2.0 ** -8)) == one
    # 1 + 3 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: the even one is 1 + 2^-6
    assert oracle.bf16_round(np.float32(1 + 3 * 2.0 ** -8)) == np.float32(1 + 2.0 ** -6)
    assert oracle.bf16_round(np.float32(1 + 2.0 ** -8 + 2.0 ** -20)) == np.float32(1 + 2.0 ** -7)
    assert oracle.bf16_round(np.float32(-1 - 2.0 ** -8)) == -one
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-6, 6, 20000),
                        (rng.integers(-2 ** 15, 2 ** 15, 2000) * 2.0 ** -15).astype(np.float32) + np.float32(2.0 ** -24)])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.bf16_round(a), ref)


def test_bf16_form_costs_reduce_to_euclidean_on_bf16_frames():
    """Frames that BF16 holds exactly: |x|^2 + |y|^2 - 2 x.y = |x - y|^2, so the
    form's costs are the Euclidean costs of Section 4.1 (up to FP64 rounding)."""
    rng = np.random.default_rng(12)
    X = oracle.bf16_round(rng.standard_normal((9, 64)).astype(np.float32))
    Y = oracle.bf16_round(rng.standard_normal((7, 64)).astype(np.float32))
    Y[3] = X[2]  # an identical frame: the clamp at 0 holds the cost at exactly 0
    C = oracle.bf16_form_costs(X, Y)
    ref = np.array(brute.cost_table(X, Y))
    assert np.allclose(C, ref, rtol=1e-12, atol=1e-6)
    assert C[2, 3] == 0.0 or C[2, 3] < 1e-6


def test_bf16_form_costs_handworked():
    """d = 1, x = 1 + 2^-9, y = 1: the norms come from the FP32 frames,
    (1 + 2^-9)^2 and 1; the dot product from the BF16 frames, 1 * 1 (1 + 2^-9
    rounds to 1).  Cost = sqrt(2^-8 + 2^-18), not 2^-9 (an FP32 dot product)
    nor 0 (norms of the rounded frames)."""
    X = np.array([[1 + 2.0 ** -9]], np.float32)
    Y = np.array([[1.0]], np.float32)
    C = oracle.bf16_form_costs(X, Y)
    assert C[0, 0] == pytest.approx(math.sqrt(2.0 ** -8 + 2.0 ** -18), rel=1e-12)
    # swapped roles give the same cost
    assert oracle.bf16_form_costs(Y, X)[0, 0] == C[0, 0]
