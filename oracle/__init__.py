"""CPU oracle for exact DTW alignment -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  The product path
never does, and this package imports nothing from the product package.

Wraps ``dtw_oracle.c`` (plain C, FP64 / int64):

* :func:`dtw`       -- oracle 1, textbook DTW with backpointers and backtrace
                       (Section 2.1, Eq. "recurrence" and Eq. "dtwboundary"),
                       ties broken DIAG, then UP, then LEFT.
* :func:`linmdtw`   -- oracle 2, the divide-and-conquer linear-memory alignment
                       (Algorithm 2 with Algorithm 1 as its sweep), counting
                       processed cells (Section 3.2).
* :func:`acc_matrix`-- whole forward D or backward B matrix (small cases), for
                       the split-cost identity of Lemma 2.
* :func:`path_cost` -- sum of C along a path (re-scoring in FP64 / int64).
* :func:`edit`      -- weighted edit distance (Section 5 names it as a problem of
                       the same DP design): its plain definition over the node
                       grid with a pointer per node (ties DIAG, UP, LEFT) and a
                       backtrace (``edit_oracle.c``).
* :func:`edit_table`-- the whole edit-distance table, forward or of the reversed
                       sequences (the recursion's split identity).
* :func:`local`     -- local alignment (Smith-Waterman, named in Section 5 beside
                       edit distance): score, the canonical end, start and path
                       (``edit_oracle.c`` states the definition).
* :func:`dtw_given` -- oracle 1 on an explicit FP64 cost matrix (the textbook DP
                       and backtrace unchanged; only C(i, j) is supplied).
* :func:`bf16_round` / :func:`bf16_form_costs` -- the cost matrix of the BF16
                       tensor-core form: the Euclidean cost of Section 4.1 in its
                       expanded form sqrt(max(0, |x|^2 + |y|^2 - 2 x.y)), with the
                       dot product taken over the frames rounded to BF16 (round to
                       nearest, ties to even) and everything else in FP64.
* :func:`path_discrepancy` -- the alignment discrepancy of two warping paths
                       (Section 4.3, Results): per cell of the first path, its
                       distance along its row and along its column to the
                       second path (plain Python over the cells; small paths).

Parity status: every function here is pinned by ``tests/test_oracle.py``
against brute-force enumeration, closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "dtw_oracle.c"), os.path.join(_HERE, "edit_oracle.c"), os.path.join(_HERE, "oracle_impl.h")]

EUCLID_F32 = 0
ABS_I32 = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add) if it is stale."""
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in _SRC)
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-Wall", "-ffp-contract=off", "-shared", "-fPIC",
             _SRC[0], _SRC[1], "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.oracle_dtw.argtypes = [p, i64, p, i64, i32, i32, p, p, p, p]
        lib.oracle_linmdtw.argtypes = [p, i64, p, i64, i32, i32, i64, p, p, p, p, p]
        lib.oracle_acc_matrix.argtypes = [p, i64, p, i64, i32, i32, i32, p, p]
        lib.oracle_path_cost.argtypes = [p, i64, p, i64, i32, i32, p, i64, p, p]
        lib.oracle_edit.argtypes = [p, i64, p, i64, i64, i64, p, p, p]
        lib.oracle_edit_table.argtypes = [p, i64, p, i64, i64, i64, i32, p]
        lib.oracle_local.argtypes = [p, i64, p, i64, i64, i64, i64, p, p, p, p]
        lib.oracle_dtw_given.argtypes = [p, i64, i64, p, p, p]
        for f in (lib.oracle_dtw_given, lib.oracle_dtw, lib.oracle_linmdtw, lib.oracle_acc_matrix, lib.oracle_path_cost, lib.oracle_edit,
                  lib.oracle_edit_table, lib.oracle_local):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _prep(X, Y):
    """Returns contiguous (X, Y, M, N, d, kind) from 1-D/2-D float32 or int32 arrays."""
    X = np.asarray(X)
    Y = np.asarray(Y)
    if X.dtype != Y.dtype:
        raise TypeError("X and Y must share a dtype")
    if X.dtype == np.int32:
        kind = ABS_I32
        X = np.ascontiguousarray(X.reshape(-1))
        Y = np.ascontiguousarray(Y.reshape(-1))
        d = 1
    elif X.dtype == np.float32:
        kind = EUCLID_F32
        if X.ndim == 1:
            X = X[:, None]
        if Y.ndim == 1:
            Y = Y[:, None]
        X = np.ascontiguousarray(X)
        Y = np.ascontiguousarray(Y)
        if X.shape[1] != Y.shape[1]:
            raise ValueError("feature dimensions differ")
        d = X.shape[1]
    else:
        raise TypeError("features must be float32 (Euclidean) or int32 (|x-y|)")
    return X, Y, X.shape[0], Y.shape[0], d, kind


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cost(kind, c, ci):
    return int(ci.value) if kind == ABS_I32 else float(c.value)


def dtw(X, Y):
    """Oracle 1.  Returns (path as int32 array of shape (K, 2), optimal cost).

    The cost is an ``int`` for int32 inputs (exact int64 sum) and a ``float``
    (FP64) for float32 inputs."""
    X, Y, M, N, d, kind = _prep(X, Y)
    path = np.empty((M + N - 1, 2), dtype=np.int32)
    K, c, ci = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    rc = _L().oracle_dtw(_ptr(X), M, _ptr(Y), N, d, kind, _ptr(path), ctypes.byref(K),
                         ctypes.byref(c), ctypes.byref(ci))
    if rc != 0:
        raise RuntimeError(f"oracle_dtw failed: {rc}")
    return path[:K.value].copy(), _cost(kind, c, ci)


def dtw_given(C):
    """Oracle 1 on a given cost matrix C (M x N, converted to FP64): returns
    (path as int32 (K, 2), optimal cost)."""
    C = np.ascontiguousarray(np.asarray(C, dtype=np.float64))
    if C.ndim != 2 or C.shape[0] < 1 or C.shape[1] < 1:
        raise ValueError("C must be a non-empty 2-D matrix")
    M, N = C.shape
    path = np.empty((M + N - 1, 2), dtype=np.int32)
    K, c = ctypes.c_int64(), ctypes.c_double()
    rc = _L().oracle_dtw_given(_ptr(C), M, N, _ptr(path), ctypes.byref(K), ctypes.byref(c))
    if rc != 0:
        raise RuntimeError(f"oracle_dtw_given failed: {rc}")
    return path[:K.value].copy(), float(c.value)


def bf16_round(a):
    """FP32 values rounded to BF16 (the upper 16 bits of the FP32 encoding: 8
    significant bits), round to nearest with ties to even, returned as FP32.
    Finite inputs only."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1  # ties go to the even upper half
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def bf16_form_costs(X, Y):
    """The BF16 form's M x N cost matrix in FP64: squared norms of the FP32
    frames, the dot product of their BF16 roundings, then
    sqrt(max(0, |x|^2 + |y|^2 - 2 x.y)) (the clamp guards the cancellation of
    near-identical frames)."""
    X = np.asarray(X, dtype=np.float32)
    Y = np.asarray(Y, dtype=np.float32)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    xx = (X64 * X64).sum(axis=1)
    yy = (Y64 * Y64).sum(axis=1)
    dot = bf16_round(X).astype(np.float64) @ bf16_round(Y).astype(np.float64).T
    return np.sqrt(np.maximum(0.0, xx[:, None] + yy[None, :] - 2.0 * dot))


def linmdtw(X, Y, m: int = 500):
    """Oracle 2 (Algorithm 2).  Returns (path, cost of that path, processed cells)."""
    X, Y, M, N, d, kind = _prep(X, Y)
    path = np.empty((M + N - 1, 2), dtype=np.int32)
    K, c, ci, cells = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    rc = _L().oracle_linmdtw(_ptr(X), M, _ptr(Y), N, d, kind, int(m), _ptr(path), ctypes.byref(K),
                             ctypes.byref(c), ctypes.byref(ci), ctypes.byref(cells))
    if rc != 0:
        raise RuntimeError(f"oracle_linmdtw failed: {rc}")
    return path[:K.value].copy(), _cost(kind, c, ci), int(cells.value)


def acc_matrix(X, Y, reverse: bool = False):
    """Whole forward D (reverse=False) or backward B (reverse=True) matrix."""
    X, Y, M, N, d, kind = _prep(X, Y)
    if kind == ABS_I32:
        out = np.empty((M, N), dtype=np.int64)
        rc = _L().oracle_acc_matrix(_ptr(X), M, _ptr(Y), N, d, kind, int(reverse), None, _ptr(out))
    else:
        out = np.empty((M, N), dtype=np.float64)
        rc = _L().oracle_acc_matrix(_ptr(X), M, _ptr(Y), N, d, kind, int(reverse), _ptr(out), None)
    if rc != 0:
        raise RuntimeError(f"oracle_acc_matrix failed: {rc}")
    return out


def path_cost(X, Y, path):
    """Sum of C(i, j) over the (K, 2) array of path cells, in path order."""
    X, Y, M, N, d, kind = _prep(X, Y)
    path = np.ascontiguousarray(np.asarray(path, dtype=np.int32).reshape(-1, 2))
    c, ci = ctypes.c_double(), ctypes.c_int64()
    rc = _L().oracle_path_cost(_ptr(X), M, _ptr(Y), N, d, kind, _ptr(path), path.shape[0],
                               ctypes.byref(c), ctypes.byref(ci))
    if rc != 0:
        raise RuntimeError(f"oracle_path_cost failed: {rc}")
    return _cost(kind, c, ci)


def path_discrepancy(P1, P2):
    """Section 4.3 (Results): for every cell (i, j) of path P1, the row error is
    min |j - k| over the cells (i, k) of path P2, and the column error is
    min |i - k| over the cells (k, j) of P2.  Returns (row_errors, col_errors),
    int64 arrays in P1's order.  Written from the definition: every P2 cell of
    the row (column) is compared; a row or column P2 never visits gives -1."""
    P1 = np.asarray(P1, dtype=np.int64).reshape(-1, 2)
    P2 = np.asarray(P2, dtype=np.int64).reshape(-1, 2)
    by_row, by_col = {}, {}
    for i, k in P2:
        by_row.setdefault(int(i), []).append(int(k))
        by_col.setdefault(int(k), []).append(int(i))
    row_err = np.empty(len(P1), dtype=np.int64)
    col_err = np.empty(len(P1), dtype=np.int64)
    for t, (i, j) in enumerate(P1):
        ks = by_row.get(int(i))
        row_err[t] = min(abs(int(j) - k) for k in ks) if ks else -1
        ks = by_col.get(int(j))
        col_err[t] = min(abs(int(i) - k) for k in ks) if ks else -1
    return row_err, col_err


def _int_seq(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))
    if a.size < 1:
        raise ValueError("empty sequence")
    return a


def edit(X, Y, sub: int = 1, gap: int = 1):
    """Weighted edit distance of int32 symbol sequences (Section 5): returns
    (path of nodes (a, b) from (0, 0) to (M, N), int32 (K, 2); optimal cost)."""
    X, Y = _int_seq(X), _int_seq(Y)
    M, N = len(X), len(Y)
    path = np.empty((M + N + 1, 2), dtype=np.int32)
    K, c = ctypes.c_int64(), ctypes.c_int64()
    rc = _L().oracle_edit(_ptr(X), M, _ptr(Y), N, int(sub), int(gap), _ptr(path), ctypes.byref(K), ctypes.byref(c))
    if rc != 0:
        raise RuntimeError(f"oracle_edit failed: {rc}")
    return path[:K.value].copy(), int(c.value)


def edit_table(X, Y, sub: int = 1, gap: int = 1, reverse: bool = False):
    """The (M+1) x (N+1) edit-distance table E (reverse: of the reversed sequences)."""
    X, Y = _int_seq(X), _int_seq(Y)
    M, N = len(X), len(Y)
    out = np.empty((M + 1, N + 1), dtype=np.int64)
    rc = _L().oracle_edit_table(_ptr(X), M, _ptr(Y), N, int(sub), int(gap), int(reverse), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle_edit_table failed: {rc}")
    return out


def edit_path_cost(X, Y, path, sub: int = 1, gap: int = 1):
    """Sum of the edge costs along a node path (DIAG: 0 or sub, UP/LEFT: gap)."""
    X, Y = _int_seq(X), _int_seq(Y)
    P = np.asarray(path, dtype=np.int64).reshape(-1, 2)
    total = 0
    for (a0, b0), (a1, b1) in zip(P[:-1], P[1:]):
        if a1 == a0 + 1 and b1 == b0 + 1:
            total += 0 if X[a1 - 1] == Y[b1 - 1] else sub
        else:
            total += gap
    return int(total)


def local(X, Y, match: int = 2, mismatch: int = 1, gap: int = 1):
    """Local alignment of int32 symbol sequences (scores +match, -mismatch,
    -gap): returns (node path (K, 2) from the start to the end node, empty when
    the score is 0; score; (a_s, b_s, a_e, b_e))."""
    X, Y = _int_seq(X), _int_seq(Y)
    M, N = len(X), len(Y)
    path = np.empty((M + N + 1, 2), dtype=np.int32)
    K, sc = ctypes.c_int64(), ctypes.c_int64()
    se = np.zeros(4, dtype=np.int64)
    rc = _L().oracle_local(_ptr(X), M, _ptr(Y), N, int(match), int(mismatch), int(gap), _ptr(path),
                           ctypes.byref(K), ctypes.byref(sc), _ptr(se))
    if rc != 0:
        raise RuntimeError(f"oracle_local failed: {rc}")
    return path[:K.value].copy(), int(sc.value), tuple(int(v) for v in se)
