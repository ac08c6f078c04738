"""Pins of the edit-distance oracle (Section 5's edit distance, weighted
Levenshtein) to things other than itself, without a GPU:

* hand-derived tables, costs and paths (tests/golden/edit_handworked.txt);
* brute force over every node path for tiny inputs: the optimum, and the
  canonical path as the lexicographically smallest backward move sequence;
* closed forms: identical sequences (0, the diagonal), disjoint alphabets;
* metric properties for S <= 2G: symmetry and the triangle inequality;
* the split identity the recursion uses: on every row a, the minimum over b of
  E(a, b) + E_R(M - a, N - b) is the optimum, and the path's cells attain it;
* the path's edge costs sum to the optimum.
"""
import os

import numpy as np
import pytest

import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "edit_handworked.txt")


def _cases():
    with open(GOLDEN) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                name, S, G, X, Y, E, cost, path = ln.split("|")
                yield (name, int(S), int(G), [int(v) for v in X.split(",")], [int(v) for v in Y.split(",")],
                       [[int(v) for v in r.split(",")] for r in E.split(";")], int(cost),
                       [tuple(int(v) for v in c.split(",")) for c in path.split(";")])


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_handworked(case):
    name, S, G, X, Y, E, cost, path = case
    assert oracle.edit_table(X, Y, S, G).tolist() == E
    p, c = oracle.edit(X, Y, S, G)
    assert c == cost
    assert [tuple(r) for r in p.tolist()] == path


def test_path_counts_match_delannoy():
    for M in range(1, 5):
        for N in range(1, 5):
            assert len(brute.edit_all_paths(M, N)) == brute.delannoy(M, N)


@pytest.mark.parametrize("alphabet,S,G", [(2, 1, 1), (3, 1, 1), (2, 2, 1), (4, 3, 2), (2, 1, 3)])
def test_vs_brute_force(alphabet, S, G):
    rng = np.random.default_rng(alphabet * 100 + S * 10 + G)
    for _ in range(40):
        M, N = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        X = rng.integers(0, alphabet, M).tolist()
        Y = rng.integers(0, alphabet, N).tolist()
        best, canon = brute.edit_solve(X, Y, S, G)
        p, c = oracle.edit(X, Y, S, G)
        assert c == best
        assert [tuple(r) for r in p.tolist()] == canon


@pytest.mark.parametrize("M", [1, 7, 50])
def test_identical_sequences(M):
    X = np.arange(M) % 5
    p, c = oracle.edit(X, X, 1, 1)
    assert c == 0
    assert p.tolist() == [[k, k] for k in range(M + 1)]


@pytest.mark.parametrize("M,N,S,G", [(5, 8, 1, 1), (9, 3, 3, 1), (4, 4, 1, 2), (12, 7, 5, 2)])
def test_disjoint_alphabets(M, N, S, G):
    """No symbol matches: min(M, N) substitutions (or deletion + insertion pairs,
    whichever is cheaper) and |M - N| gaps."""
    X, Y = np.arange(M) % 3, 10 + np.arange(N) % 4
    assert oracle.edit(X, Y, S, G)[1] == min(M, N) * min(S, 2 * G) + abs(M - N) * G


def test_metric_properties():
    rng = np.random.default_rng(11)
    for _ in range(30):
        a, b, c = (rng.integers(0, 3, int(rng.integers(1, 15))) for _ in range(3))
        for S, G in ((1, 1), (2, 1), (3, 2)):
            ab, ba = oracle.edit(a, b, S, G)[1], oracle.edit(b, a, S, G)[1]
            assert ab == ba
            assert oracle.edit(a, c, S, G)[1] <= ab + oracle.edit(b, c, S, G)[1]


@pytest.mark.parametrize("seed", range(4))
def test_split_identity_and_path(seed):
    rng = np.random.default_rng(seed)
    M, N = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    X, Y = rng.integers(0, 3, M), rng.integers(0, 3, N)
    S, G = (1, 1) if seed % 2 == 0 else (2, 1)
    E = oracle.edit_table(X, Y, S, G)
    ER = oracle.edit_table(X, Y, S, G, reverse=True)
    p, c = oracle.edit(X, Y, S, G)
    assert c == E[M, N] == ER[M, N]
    for a in range(M + 1):
        through = E[a, :] + ER[M - a, ::-1]
        assert through.min() == c
    for a, b in p:
        assert E[a, b] + ER[M - a, N - b] == c
    assert oracle.edit_path_cost(X, Y, p, S, G) == c
    steps = np.diff(p, axis=0)
    assert p[0].tolist() == [0, 0] and p[-1].tolist() == [M, N]
    assert all(tuple(s) in ((1, 1), (1, 0), (0, 1)) for s in steps)


# ---------------------------------------------------------------- local alignment
# (Smith-Waterman, named in Section 5 beside edit distance): pins of oracle.local


@pytest.mark.parametrize("alphabet,MA,MM,G", [(2, 2, 1, 1), (3, 2, 1, 1), (3, 3, 2, 2), (4, 1, 1, 1), (2, 5, 3, 1)])
def test_local_vs_brute_force(alphabet, MA, MM, G):
    rng = np.random.default_rng(alphabet * 1000 + MA * 100 + MM * 10 + G)
    for _ in range(25):
        M, N = int(rng.integers(1, 5)), int(rng.integers(1, 5))
        X = rng.integers(0, alphabet, M).tolist()
        Y = rng.integers(0, alphabet, N).tolist()
        S, se, path = brute.local_solve(X, Y, MA, MM, G)
        p, sc, se_o = oracle.local(X, Y, MA, MM, G)
        assert sc == S
        if S == 0:
            assert len(p) == 0
        else:
            assert se_o == se
            assert [tuple(r) for r in p.tolist()] == path


def test_local_closed_forms():
    # identical sequences: the whole diagonal
    X = [3, 1, 4, 1, 5, 9, 2, 6]
    p, sc, se = oracle.local(X, X, 2, 1, 1)
    assert sc == 2 * len(X) and se == (0, 0, len(X), len(X))
    assert p.tolist() == [[k, k] for k in range(len(X) + 1)]
    # no common symbol: score 0, empty alignment
    p, sc, se = oracle.local([1, 2, 3], [4, 5], 2, 1, 1)
    assert sc == 0 and len(p) == 0
    # a single common symbol: one match step
    p, sc, se = oracle.local([5, 1, 1], [2, 2, 5], 2, 1, 1)
    assert sc == 2 and se == (0, 2, 1, 3) and p.tolist() == [[0, 2], [1, 3]]


def test_local_properties():
    rng = np.random.default_rng(5)
    for _ in range(30):
        X = rng.integers(0, 4, int(rng.integers(1, 40)))
        Y = rng.integers(0, 4, int(rng.integers(1, 40)))
        p, sc, se = oracle.local(X, Y, 2, 1, 1)
        assert sc == oracle.local(Y, X, 2, 1, 1)[1]
        assert sc >= (2 if set(X.tolist()) & set(Y.tolist()) else 0)
        if sc:
            assert p[0].tolist() == [se[0], se[1]] and p[-1].tolist() == [se[2], se[3]]
            assert brute.local_path_score(X, Y, [tuple(r) for r in p.tolist()], 2, 1, 1) == sc
