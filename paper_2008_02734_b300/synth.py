"""Seeded synthetic inputs shaped like the paper's audio features.

The paper aligns orchestral recordings with chroma-like (DLNC0 + CENS, 12-d) and
MFCC-like ("mfcc-mod", high-dimensional) features at about 43 frames/s
(Section 4.1).  That dataset is not available here, so these generators make
stand-ins of the same shape: a smooth nonnegative L2-normalised 12-d walk, a
Gaussian AR(1) MFCC-like sequence whose per-dimension spread decays with the
coefficient index, and integer sequences for the bit-exact |x-y| cost.  The second
sequence of a pair is the first one resampled by a seeded random monotone warp
plus noise.

This module holds no part of the alignment method: it only draws inputs, and it is
shared by the tests, the benchmark and the oracle checks.  All arrays are
C-contiguous numpy arrays (float32 for Euclidean features, int32 for |x-y|).
"""
from __future__ import annotations

import dataclasses

import numpy as np

CHROMA_D = 12
MFCC_D = 64


def monotone_warp(rng: np.random.Generator, M: int, N: int) -> np.ndarray:
    """N nondecreasing positions in [0, M-1], first 0 and last M-1.

    Cumulative sum of Gamma(shape 4) increments, rescaled onto [0, M-1]: a smooth
    random tempo curve."""
    if N == 1:
        return np.zeros(1)
    inc = rng.gamma(4.0, 1.0, size=N - 1)
    w = np.concatenate([[0.0], np.cumsum(inc)])
    return w / w[-1] * (M - 1)


def _resample(X: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Linear interpolation of the rows of X at fractional positions w."""
    lo = np.floor(w).astype(np.int64)
    hi = np.minimum(lo + 1, X.shape[0] - 1)
    t = (w - lo)[:, None]
    return (1.0 - t) * X[lo] + t * X[hi]


def _l2_rows(A: np.ndarray) -> np.ndarray:
    n = np.linalg.norm(A, axis=1, keepdims=True)
    return A / np.maximum(n, 1e-12)


def chroma_walk(rng: np.random.Generator, M: int, d: int = CHROMA_D) -> np.ndarray:
    """Smooth nonnegative random walk v_{t+1} = |v_t + N(0, 0.05^2)|, rows L2-normalised."""
    v = np.empty((M, d))
    v[0] = np.abs(rng.standard_normal(d))
    steps = rng.normal(0.0, 0.05, size=(M, d))
    for t in range(1, M):
        v[t] = np.abs(v[t - 1] + steps[t])
    return _l2_rows(v).astype(np.float32)


def chroma_pair(seed: int, M: int, N: int, noise: float = 0.05):
    """Chroma-like pair: X is a walk of M frames; Y is X warped to N frames plus
    Gaussian noise, clipped at 0 and renormalised."""
    rng = np.random.default_rng(seed)
    X = chroma_walk(rng, M)
    w = monotone_warp(rng, M, N)
    Y = _resample(X.astype(np.float64), w) + rng.normal(0.0, noise, size=(N, X.shape[1]))
    Y = _l2_rows(np.maximum(Y, 0.0)).astype(np.float32)
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def mfcc_like(rng: np.random.Generator, M: int, d: int = MFCC_D, rho: float = 0.9) -> np.ndarray:
    """Gaussian AR(1) per dimension, mean 0, stationary std 1/(1+k/8) for dim k."""
    sd = 1.0 / (1.0 + np.arange(d) / 8.0)
    z = np.empty((M, d))
    z[0] = rng.standard_normal(d)
    e = rng.standard_normal((M, d)) * np.sqrt(1.0 - rho * rho)
    for t in range(1, M):
        z[t] = rho * z[t - 1] + e[t]
    return (z * sd).astype(np.float32)


def mfcc_pair(seed: int, M: int, N: int, d: int = MFCC_D, noise: float = 0.1):
    """MFCC-like pair: X is AR(1) frames; Y is X warped to N frames plus N(0, noise^2)."""
    rng = np.random.default_rng(seed)
    X = mfcc_like(rng, M, d)
    w = monotone_warp(rng, M, N)
    Y = _resample(X.astype(np.float64), w) + rng.normal(0.0, noise, size=(N, d))
    return np.ascontiguousarray(X), np.ascontiguousarray(Y.astype(np.float32))


def int_pair(seed: int, M: int, N: int, lo: int = 0, hi: int = 255, noise: int = 8):
    """Integer pair: X uniform in [lo, hi]; Y is X at the nearest warped index plus
    integer noise uniform in [-noise, noise] (not clipped)."""
    rng = np.random.default_rng(seed)
    X = rng.integers(lo, hi + 1, size=M, dtype=np.int64)
    w = monotone_warp(rng, M, N)
    Y = X[np.rint(w).astype(np.int64)] + rng.integers(-noise, noise + 1, size=N)
    return X.astype(np.int32), Y.astype(np.int32)


# ---------------------------------------------------------------------------
# The five workloads (sizes and distributions as the benchmark configurations)
# ---------------------------------------------------------------------------

def workload_plain_float(seed: int = 0):
    """2000 x 12-d chroma-like FP32 frames vs a 2500-frame warped, noisy copy."""
    return chroma_pair(seed, 2000, 2500)


def workload_int_pair(seed: int = 1, M: int = 20000, N: int = 24000):
    """1-D int32 pair, M=20000, N=24000, values in [0,255], noise in [-8,8]."""
    return int_pair(seed, M, N)


def workload_precision(seed: int = 2, M: int = 60000, N: int = 75000):
    """60000 x 64-d MFCC-like frames vs a 75000-frame warp plus sigma=0.1 noise."""
    return mfcc_pair(seed, M, N)


def _log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))


def workload_batch_sizes(seed: int = 3, B: int = 256, lo: int = 1000, hi: int = 20000):
    """(M, N) of the uneven batch: M log-uniform in [lo, hi], ratio r log-uniform in
    [0.8, 1.25], N = clip(round(r M), lo, hi)."""
    rng = np.random.default_rng(seed)
    M = np.rint(_log_uniform(rng, lo, hi, B)).astype(np.int64)
    r = _log_uniform(rng, 0.8, 1.25, B)
    N = np.clip(np.rint(r * M), lo, hi).astype(np.int64)
    return M, N


def batch_pair(k: int, seed: int = 3, B: int = 256, lo: int = 1000, hi: int = 20000):
    """Pair k of the uneven chroma-like batch (as workload_batch builds it)."""
    M, N = workload_batch_sizes(seed, B, lo, hi)
    return chroma_pair(seed * 100003 + k, int(M[k]), int(N[k]))


def workload_batch(seed: int = 3, B: int = 256, lo: int = 1000, hi: int = 20000):
    """The uneven batch of chroma-like pairs: list of (X, Y)."""
    M, N = workload_batch_sizes(seed, B, lo, hi)
    return [chroma_pair(seed * 100003 + k, int(M[k]), int(N[k])) for k in range(B)]


def batch_int_pair(k: int, seed: int = 3, B: int = 256, lo: int = 1000, hi: int = 20000):
    """Pair k of the uneven batch's integer counterpart: the same (M, N) with
    int_pair data (values in [0, 255], noise in [-8, 8])."""
    M, N = workload_batch_sizes(seed, B, lo, hi)
    return int_pair(seed * 100003 + k, int(M[k]), int(N[k]))


def workload_batch_int(seed: int = 3, B: int = 256, lo: int = 1000, hi: int = 20000):
    """The uneven batch's shapes with 1-D int32 |x-y| data: list of (X, Y)."""
    return [batch_int_pair(k, seed, B, lo, hi) for k in range(B)]


@dataclasses.dataclass
class Request:
    arrival_s: float
    M: int
    N: int
    d: int
    seed: int

    def features(self):
        if self.d == CHROMA_D:
            return chroma_pair(self.seed, self.M, self.N)
        return mfcc_pair(self.seed, self.M, self.N, self.d)


def workload_serving(seed: int = 4, R: int = 2000, rate_hz: float = 100.0,
                     lo: int = 500, hi: int = 100000):
    """Poisson arrivals of R requests; lengths log-uniform in [lo, hi], ratio as the
    batch, feature dimension 12 or 64 with equal probability."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=R)
    t = np.cumsum(gaps) - gaps[0]
    M = np.rint(_log_uniform(rng, lo, hi, R)).astype(np.int64)
    r = _log_uniform(rng, 0.8, 1.25, R)
    N = np.clip(np.rint(r * M), lo, hi).astype(np.int64)
    d = np.where(rng.random(R) < 0.5, CHROMA_D, MFCC_D)
    return [Request(float(t[k]), int(M[k]), int(N[k]), int(d[k]), seed * 1000003 + k)
            for k in range(R)]


def edit_pair(seed: int, M: int, rate: float = 0.1, alphabet: int = 4):
    """Symbol sequences for edit distance: X uniform over ``alphabet`` symbols; Y
    is X after random point mutations -- at each position, with probability
    ``rate``, a substitution, a deletion or an insertion (equally likely)."""
    rng = np.random.default_rng(seed)
    X = rng.integers(0, alphabet, M).astype(np.int32)
    out = []
    for v in X:
        if rng.random() < rate:
            kind = rng.integers(3)
            if kind == 0:
                out.append(int(rng.integers(0, alphabet)))
            elif kind == 2:
                out.append(int(v))
                out.append(int(rng.integers(0, alphabet)))
            # kind == 1: deletion
        else:
            out.append(int(v))
    if not out:
        out.append(int(rng.integers(0, alphabet)))
    return X, np.asarray(out, dtype=np.int32)


def workload_edit_pair(seed: int = 4, M: int = 20000):
    """A 20000-symbol sequence over 4 symbols against a 10%-mutated copy."""
    return edit_pair(seed, M)


def local_pair(seed: int, M: int, N: int, core: int, rate: float = 0.1, alphabet: int = 4):
    """Sequences for local alignment: X and Y uniform over ``alphabet`` symbols,
    with a ``core``-symbol stretch of X planted, after point mutations (as in
    edit_pair), at a random place in Y."""
    rng = np.random.default_rng(seed)
    X = rng.integers(0, alphabet, M).astype(np.int32)
    Y = rng.integers(0, alphabet, N).astype(np.int32)
    core = max(1, min(core, M, N // 2))
    i0 = int(rng.integers(0, M - core + 1))
    mut = []
    for v in X[i0:i0 + core]:
        if rng.random() < rate:
            kind = rng.integers(3)
            if kind == 0:
                mut.append(int(rng.integers(0, alphabet)))
            elif kind == 2:
                mut.append(int(v))
                mut.append(int(rng.integers(0, alphabet)))
        else:
            mut.append(int(v))
    mut = np.asarray(mut[: N], dtype=np.int32)
    j0 = int(rng.integers(0, N - len(mut) + 1))
    Y[j0:j0 + len(mut)] = mut
    return X, Y


def workload_local_pair(seed: int = 5):
    """20000 vs 24000 random symbols sharing a mutated 5000-symbol stretch."""
    return local_pair(seed, 20000, 24000, 5000)
