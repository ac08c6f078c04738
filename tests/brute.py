"""Brute-force DTW by enumerating every warping path (tiny inputs only).

Independent of the oracle and of the CUDA path: the frame cost is evaluated here
in plain Python (double, dims in ascending order, correctly rounded sqrt), and a
path's cost is its cost terms summed from the first cell to the last.

A warping path (Section 2.1) starts at (0,0), ends at (M-1,N-1) and advances by
(0,1), (1,0) or (1,1).  Among all optimal paths, the "canonical" one is the path
whose sequence of moves, read backward from (M-1,N-1), is lexicographically
smallest with DIAG < UP < LEFT -- the path a backtrace yields when each
backpointer is the first minimum in the order DIAG, UP, LEFT.
"""
from __future__ import annotations

import math
from math import comb

DIAG, UP, LEFT = 0, 1, 2


def frame_cost(x, y):
    if isinstance(x, (int,)) or (hasattr(x, "dtype") and x.dtype.kind == "i" and x.ndim == 0):
        return abs(int(x) - int(y))
    s = 0.0
    for a, b in zip(x, y):
        t = float(a) - float(b)
        s = s + t * t
    return math.sqrt(s)


def cost_table(X, Y):
    return [[frame_cost(X[i], Y[j]) for j in range(len(Y))] for i in range(len(X))]


def all_paths(M, N):
    """Every warping path from (0,0) to (M-1,N-1), as lists of cells."""
    out = []

    def rec(i, j, acc):
        acc.append((i, j))
        if i == M - 1 and j == N - 1:
            out.append(list(acc))
        else:
            if j + 1 < N:
                rec(i, j + 1, acc)
            if i + 1 < M:
                rec(i + 1, j, acc)
            if i + 1 < M and j + 1 < N:
                rec(i + 1, j + 1, acc)
        acc.pop()

    rec(0, 0, [])
    return out


def delannoy(m, n):
    """Closed form for the number of lattice paths with steps E, N, NE."""
    return sum(comb(m, k) * comb(n, k) * (1 << k) for k in range(min(m, n) + 1))


def backward_moves(path):
    mv = []
    for (i1, j1), (i0, j0) in zip(path[:0:-1], path[-2::-1]):
        if i1 - i0 == 1 and j1 - j0 == 1:
            mv.append(DIAG)
        elif i1 - i0 == 1:
            mv.append(UP)
        else:
            mv.append(LEFT)
    return tuple(mv)


def solve(X, Y):
    """(optimal cost, canonical path, number of optimal paths, number of paths)."""
    return solve_table(cost_table(X, Y))


def solve_table(C):
    """solve() over a given cost table C (a list of rows, or a 2-D array)."""
    M, N = len(C), len(C[0])
    C = [[float(v) if not isinstance(v, int) else v for v in row] for row in C]
    best = None
    opt = []
    paths = all_paths(M, N)
    for p in paths:
        s = 0
        for (i, j) in p:
            s = s + C[i][j]
        if best is None or s < best:
            best = s
            opt = [p]
        elif s == best:
            opt.append(p)
    canon = min(opt, key=backward_moves)
    return best, canon, len(opt), len(paths)


def prefix_optimum(X, Y, i, j):
    """Optimal cost over warping paths from (0,0) to (i,j)."""
    return solve(X[: i + 1], Y[: j + 1])[0]


def suffix_optimum(X, Y, i, j):
    """Optimal cost over warping paths from (i,j) to (M-1,N-1), C(i,j) included,
    summed from the last cell back to (i,j)."""
    Xr, Yr = X[i:][::-1], Y[j:][::-1]
    return solve(Xr, Yr)[0]


# ---------------------------------------------------------------- edit distance

def edit_all_paths(M, N):
    """Every node path from (0, 0) to (M, N) with steps (1,1), (1,0), (0,1)."""
    out = []

    def rec(a, b, acc):
        if (a, b) == (M, N):
            out.append(list(acc))
            return
        for da, db in ((1, 1), (1, 0), (0, 1)):
            if a + da <= M and b + db <= N:
                acc.append((a + da, b + db))
                rec(a + da, b + db, acc)
                acc.pop()

    rec(0, 0, [(0, 0)])
    return out


def edit_path_cost(X, Y, path, S, G):
    total = 0
    for (a0, b0), (a1, b1) in zip(path[:-1], path[1:]):
        if a1 == a0 + 1 and b1 == b0 + 1:
            total += 0 if X[a1 - 1] == Y[b1 - 1] else S
        else:
            total += G
    return total


def edit_solve(X, Y, S, G):
    """(optimal cost, canonical path): the minimum over every node path, and among
    the optimal ones the lexicographically smallest backward move sequence with
    DIAG < UP < LEFT."""
    M, N = len(X), len(Y)
    best, cands = None, []
    for p in edit_all_paths(M, N):
        c = edit_path_cost(X, Y, p, S, G)
        if best is None or c < best:
            best, cands = c, [p]
        elif c == best:
            cands.append(p)
    return best, min(cands, key=backward_moves)


# ---------------------------------------------------------------- local alignment

def node_paths(s, e):
    """Every node path from node s to node e (steps (1,1), (1,0), (0,1))."""
    (a0, b0), (a1, b1) = s, e
    return [[(a0 + a, b0 + b) for a, b in p] for p in edit_all_paths(a1 - a0, b1 - b0)] if (a1 - a0) + (b1 - b0) else [[s]]


def local_path_score(X, Y, path, MA, MM, G):
    total = 0
    for (a0, b0), (a1, b1) in zip(path[:-1], path[1:]):
        if a1 == a0 + 1 and b1 == b0 + 1:
            total += MA if X[a1 - 1] == Y[b1 - 1] else -MM
        else:
            total -= G
    return total


def local_solve(X, Y, MA, MM, G):
    """(score, (a_s, b_s, a_e, b_e) or None, path) by enumeration: the best score
    over every pair of nodes s <= e and every node path between them; the end is
    the first node in row-major order whose best alignment ending there reaches
    the score, the start the largest node in row-major order from which a path to
    that end reaches it, the path the lexicographically smallest backward move
    sequence (DIAG < UP < LEFT) among those paths."""
    M, N = len(X), len(Y)
    nodes = [(a, b) for a in range(M + 1) for b in range(N + 1)]

    def best(s, e):
        return max(local_path_score(X, Y, p, MA, MM, G) for p in node_paths(s, e))

    H = {}
    for e in nodes:
        H[e] = max([0] + [best(s, e) for s in nodes if s[0] <= e[0] and s[1] <= e[1] and s != e])
    S = max(H.values())
    if S == 0:
        return 0, None, []
    e = min(n for n in nodes if H[n] == S)
    starts = [s for s in nodes if s[0] <= e[0] and s[1] <= e[1] and s != e and best(s, e) == S]
    s = max(starts)
    cands = [p for p in node_paths(s, e) if local_path_score(X, Y, p, MA, MM, G) == S]
    return S, (s[0], s[1], e[0], e[1]), min(cands, key=backward_moves)
