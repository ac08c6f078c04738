"""Exact linear-memory DTW alignment on B300 (sm_103a): thin Python binding.

Every function here only marshals arguments for the C ABI declared in
``include/dtw_b300.h`` and implemented in ``libdtw_b300.so`` (CUDA kernels for
the divide-and-conquer recursion of Section 3.2).  There is no Python or CPU
fallback: the first call into the library fails if it has not been built.

Inputs may be torch tensors (CPU or CUDA) or numpy arrays: float32 frames of
shape (M, d) use the Euclidean frame cost, int32 sequences of shape (M,) use
|x - y|.  CUDA inputs are aligned on the tensors' device with the current torch
stream; host inputs are staged by the library (host-to-device copy inside the
call).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libdtw_b300.so")

EUCLID_F32 = 0
ABS_I32 = 1
PLAIN_F64 = 1 << 8
COST_BF16 = 1 << 9
DP_F32_KAHAN = 1 << 10


def _form(dp_f32: bool, cost_bf16: bool) -> int:
    return (DP_F32_KAHAN if dp_f32 else 0) | (COST_BF16 if cost_bf16 else 0)

OK, PENDING, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW, EBUSY, EINTERNAL = 0, 1, -1, -2, -3, -4, -5, -6, -7
OPT_TIMING, OPT_BASE_AREA, OPT_SPIN_LIMIT, OPT_SKIP_PUBLISH, OPT_GRAPH, OPT_SWEEP_VARIANT = 1, 2, 3, 4, 5, 6
OPT_EDIT_SUB, OPT_EDIT_GAP = 7, 8
OPT_NOALLOC_EPOCH = 9  # test hook: the next dtw_cost_noalloc call's first boundary-word epoch
OPT_FUSED_SPLIT = 10  # 0 separate split launch, 1 (default) float kinds and batches in the sweep kernel, 2 always
OPT_SPLIT_WINDOWS = 11  # windows of split rows per box and level, at most (1: the paper's single split; default 7)
EDIT_I32 = 2  # weighted edit distance of int32 symbol sequences (cost kind)


class DTWError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_strerror(status)} ({status})")


class Stats(ctypes.Structure):
    _fields_ = [("problem_cells", ctypes.c_int64), ("sweep_cells", ctypes.c_int64),
                ("tag_cells", ctypes.c_int64), ("base_cells", ctypes.c_int64),
                ("levels", ctypes.c_int32), ("sweep_launches", ctypes.c_int32),
                ("base_boxes", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("retagged_boxes", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("resyncs", ctypes.c_int64), ("polls", ctypes.c_int64),
                ("sweep_ms", ctypes.c_double), ("device_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class Request(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("M", ctypes.c_int64), ("Y", ctypes.c_void_p), ("N", ctypes.c_int64),
                ("d", ctypes.c_int32), ("cost_kind", ctypes.c_int32), ("path_out", ctypes.c_void_p)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    sig = {
        "dtw_align": (i64, [vp, i64, vp, i64, i32, i32, vp, vp]),
        "dtw_cost": (ctypes.c_int, [vp, i64, vp, i64, i32, i32, vp]),
        "dtw_align_batch": (ctypes.c_int, [i32, vp, vp, vp, vp, i32, i32, vp, vp, vp]),
        "dtw_submit": (i64, [vp]),
        "dtw_poll": (ctypes.c_int, [i64, vp, vp]),
        "dtw_set_stream": (ctypes.c_int, [vp]),
        "dtw_set_budget": (ctypes.c_int, [u64]),
        "dtw_set_arena": (ctypes.c_int, [vp, u64]),
        "dtw_footprint": (ctypes.c_size_t, [i64, i64, i32, i32]),
        "dtw_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "dtw_get_stats": (ctypes.c_int, [vp]),
        "dtw_pipe_rates": (ctypes.c_int, [vp, i32]),
        "dtw_set_option": (ctypes.c_int, [i32, i64]),
        "dtw_cost_noalloc": (ctypes.c_int, [vp, i64, vp, i64, i32, i32, vp, vp]),
        "dtw_path_discrepancy": (ctypes.c_int, [vp, i64, vp, i64, i64, i64, vp, vp]),
        "dtw_local_align": (ctypes.c_int, [vp, i64, vp, i64, i32, i32, i32, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB_PATH = _LIB_PATH
_lib = None


def _get_lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def __getattr__(name):
    # the ctypes library is loaded on first use, so that ``synth`` imports without it
    if name == "lib":
        return _get_lib()
    raise AttributeError(name)

# exported names of the C ABI, for the symbol check
ABI_FUNCTIONS = ("dtw_align", "dtw_cost", "dtw_align_batch", "dtw_submit", "dtw_poll", "dtw_set_stream",
                 "dtw_set_budget", "dtw_set_arena", "dtw_footprint", "dtw_strerror", "dtw_get_stats", "dtw_pipe_rates",
                 "dtw_set_option", "dtw_cost_noalloc", "dtw_path_discrepancy", "dtw_local_align")


def _strerror(status: int) -> str:
    return _get_lib().dtw_strerror(int(status)).decode()


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise DTWError(int(rc), where)
    return rc


# ------------------------------------------------------------------ marshalling

def _as_buffer(a):
    """(object kept alive, data pointer, shape, dtype-kind, is_cuda) of a tensor or array."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                a = a.contiguous()
            kind = {torch.float32: EUCLID_F32, torch.int32: ABS_I32}.get(a.dtype)
            if kind is None:
                raise TypeError("frames must be float32 (Euclidean) or int32 (|x-y|)")
            return a, a.data_ptr(), tuple(a.shape), kind, a.is_cuda
    except ImportError:
        pass
    a = np.ascontiguousarray(a)
    kind = {np.dtype(np.float32): EUCLID_F32, np.dtype(np.int32): ABS_I32}.get(a.dtype)
    if kind is None:
        raise TypeError("frames must be float32 (Euclidean) or int32 (|x-y|)")
    return a, a.ctypes.data, a.shape, kind, False


def _dims(shape, kind):
    if kind == ABS_I32:
        if len(shape) == 2 and shape[1] != 1:
            raise ValueError("int32 sequences are 1-D")
        return shape[0], 1
    if len(shape) == 1:
        return shape[0], 1
    return shape[0], shape[1]


def _prep_pair(X, Y):
    xo, xp, xs, xk, xc = _as_buffer(X)
    yo, yp, ys, yk, yc = _as_buffer(Y)
    if xk != yk:
        raise TypeError("X and Y must have the same dtype")
    M, dx = _dims(xs, xk)
    N, dy = _dims(ys, yk)
    if dx != dy:
        raise ValueError("feature dimensions differ")
    return (xo, yo), xp, M, yp, N, dx, xk, (xc or yc), (xo if xc else yo if yc else None)


def _sync_stream(cuda_tensor):
    """Run on the tensor's device and the current torch stream."""
    import torch
    dev = cuda_tensor.device
    torch.cuda.set_device(dev)
    _get_lib().dtw_set_stream(ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))


def _path_buffer(M, N, like_cuda):
    import torch
    if like_cuda is not None:
        return torch.empty((M + N - 1, 2), dtype=torch.int32, device=like_cuda.device)
    return torch.empty((M + N - 1, 2), dtype=torch.int32)


def align(X, Y, *, plain: bool = False, dp_f32: bool = False, cost_bf16: bool = False, path_out=None):
    """Exact DTW of one pair: returns (path as an int32 tensor of shape (K, 2), D*).

    ``plain=True`` runs the paper's plain FP64 form (one launch per anti-diagonal)
    instead of the tiled path; ``dp_f32=True`` (float frames) accumulates in
    compensated FP32 pairs instead of FP64; ``cost_bf16=True`` (d = 64) uses the
    reduced-precision tensor-core cost form.  ``path_out`` may supply the
    (M+N-1, 2) int32 output buffer (host or device)."""
    keep, xp, M, yp, N, d, kind, on_cuda, cu = _prep_pair(X, Y)
    if cu is not None:
        _sync_stream(cu)
    path = _path_buffer(M, N, cu) if path_out is None else path_out
    ck = kind | (PLAIN_F64 if plain else 0) | _form(dp_f32, cost_bf16)
    cost = ctypes.c_double()
    K = _get_lib().dtw_align(xp, M, yp, N, d, ck, ctypes.c_void_p(path.data_ptr()), ctypes.byref(cost))
    _check(K, "dtw_align")
    c = cost.value
    return path[:K], (int(c) if kind == ABS_I32 else c)


def cost(X, Y, *, dp_f32: bool = False, cost_bf16: bool = False):
    """D* only (one forward sweep, no path)."""
    keep, xp, M, yp, N, d, kind, on_cuda, cu = _prep_pair(X, Y)
    if cu is not None:
        _sync_stream(cu)
    c = ctypes.c_double()
    ck = kind | _form(dp_f32, cost_bf16)
    _check(_get_lib().dtw_cost(xp, M, yp, N, d, ck, ctypes.byref(c)), "dtw_cost")
    return int(c.value) if kind == ABS_I32 else c.value


def cost_noalloc(X, Y):
    """D* through the entry point that allocates no device memory (CUDA inputs only);
    see dtw_cost_noalloc in include/dtw_b300.h for its size limits."""
    keep, xp, M, yp, N, d, kind, on_cuda, cu = _prep_pair(X, Y)
    if cu is None:
        raise ValueError("dtw_cost_noalloc needs CUDA inputs")
    import torch
    torch.cuda.set_device(cu.device)
    c = ctypes.c_double()
    st = ctypes.c_void_p(torch.cuda.current_stream(cu.device).cuda_stream)
    _check(_get_lib().dtw_cost_noalloc(xp, M, yp, N, d, kind, ctypes.byref(c), st), "dtw_cost_noalloc")
    return int(c.value) if kind == ABS_I32 else c.value


def path_discrepancy(P1, P2, M: int, N: int):
    """Alignment discrepancy of two warping paths of an M x N problem (Section
    4.3): returns (errors, max) with errors an int32 (2, K1) tensor on P1's device
    -- row 0 the row errors of P1's cells, row 1 their column errors."""
    import torch
    P1 = torch.as_tensor(P1, dtype=torch.int32).contiguous()
    P2 = torch.as_tensor(P2, dtype=torch.int32).contiguous()
    if P1.dim() != 2 or P1.shape[1] != 2 or P2.dim() != 2 or P2.shape[1] != 2:
        raise ValueError("paths are (K, 2) arrays of (i, j)")
    if P1.is_cuda:
        _sync_stream(P1)
    elif P2.is_cuda:
        _sync_stream(P2)
    err = torch.empty((2, P1.shape[0]), dtype=torch.int32, device=P1.device)
    mx = ctypes.c_int32()
    _check(_get_lib().dtw_path_discrepancy(P1.data_ptr(), P1.shape[0], P2.data_ptr(), P2.shape[0], int(M), int(N),
                                           err.data_ptr(), ctypes.byref(mx)), "dtw_path_discrepancy")
    return err, int(mx.value)


def _edit_args(X, Y, sub, gap):
    keep, xp, M, yp, N, d, kind, on_cuda, cu = _prep_pair(X, Y)
    if kind != ABS_I32 or d != 1:
        raise TypeError("edit distance takes 1-D int32 symbol sequences")
    set_option(OPT_EDIT_SUB, int(sub))
    set_option(OPT_EDIT_GAP, int(gap))
    if cu is not None:
        _sync_stream(cu)
    return keep, xp, M, yp, N, cu


def _node_path_buffer(M, N, like_cuda):
    import torch
    dev = like_cuda.device if like_cuda is not None else "cpu"
    return torch.empty((M + N + 1, 2), dtype=torch.int32, device=dev)


def edit_align(X, Y, *, sub: int = 1, gap: int = 1, path_out=None):
    """Weighted edit distance of two int32 symbol sequences through the same
    linear-memory recursion (Section 5): returns (node path, an int32 (K, 2)
    tensor from (0, 0) to (M, N); exact cost).  A DIAG step is a match (cost 0) or
    a substitution (``sub``), UP and LEFT steps are gaps (``gap``)."""
    keep, xp, M, yp, N, cu = _edit_args(X, Y, sub, gap)
    path = _node_path_buffer(M, N, cu) if path_out is None else path_out
    c = ctypes.c_double()
    K = _get_lib().dtw_align(xp, M, yp, N, 1, EDIT_I32, ctypes.c_void_p(path.data_ptr()), ctypes.byref(c))
    _check(K, "dtw_align")
    return path[:K], int(c.value)


def local_align(X, Y, *, match: int = 2, mismatch: int = 1, gap: int = 1, path_out=None):
    """Local alignment (Smith-Waterman, Section 5) of two int32 symbol sequences
    in linear memory: returns (node path from the start to the end node, an int32
    (K, 2) tensor, empty when the score is 0; score; (a_s, b_s, a_e, b_e))."""
    keep, xp, M, yp, N, d, kind, on_cuda, cu = _prep_pair(X, Y)
    if kind != ABS_I32 or d != 1:
        raise TypeError("local alignment takes 1-D int32 symbol sequences")
    if cu is not None:
        _sync_stream(cu)
    path = _node_path_buffer(M, N, cu) if path_out is None else path_out
    K, sc = ctypes.c_int64(), ctypes.c_int64()
    se = (ctypes.c_int64 * 4)()
    _check(_get_lib().dtw_local_align(xp, M, yp, N, int(match), int(mismatch), int(gap),
                                      ctypes.c_void_p(path.data_ptr()), ctypes.byref(K), ctypes.byref(sc), se),
           "dtw_local_align")
    return path[:K.value], int(sc.value), tuple(int(v) for v in se)


def edit_distance(X, Y, *, sub: int = 1, gap: int = 1) -> int:
    """The weighted edit distance only (one forward sweep of the node grid)."""
    keep, xp, M, yp, N, cu = _edit_args(X, Y, sub, gap)
    c = ctypes.c_double()
    _check(_get_lib().dtw_cost(xp, M, yp, N, 1, EDIT_I32, ctypes.byref(c)), "dtw_cost")
    return int(c.value)


def edit_align_batch(Xs, Ys, *, sub: int = 1, gap: int = 1):
    """Edit-distance alignments of B pairs together; returns a list of (node path, cost)."""
    B = len(Xs)
    if B != len(Ys) or B == 0:
        raise ValueError("need equally many, and at least one, X and Y")
    keep, xps, yps, Ms, Ns, paths = [], [], [], [], [], []
    cu0 = None
    for X, Y in zip(Xs, Ys):
        k, xp, M, yp, N, cu = _edit_args(X, Y, sub, gap)
        cu0 = cu0 if cu0 is not None else cu
        keep.append(k)
        xps.append(xp)
        yps.append(yp)
        Ms.append(M)
        Ns.append(N)
        paths.append(_node_path_buffer(M, N, cu))
    VP = ctypes.c_void_p * B
    I64 = ctypes.c_int64 * B
    K = I64()
    C = (ctypes.c_double * B)()
    rc = _get_lib().dtw_align_batch(B, VP(*xps), I64(*Ms), VP(*yps), I64(*Ns), 1, EDIT_I32,
                                    VP(*[p.data_ptr() for p in paths]), K, C)
    _check(rc, "dtw_align_batch")
    return [(paths[b][:K[b]], int(C[b])) for b in range(B)]


def align_batch(Xs, Ys, *, dp_f32: bool = False, cost_bf16: bool = False, paths_out=None):
    """Aligns B pairs together; returns a list of (path, D*).  ``paths_out`` may
    supply the B (M+N-1, 2) int32 output buffers (host or device)."""
    B = len(Xs)
    if B != len(Ys) or B == 0:
        raise ValueError("need equally many, and at least one, X and Y")
    keep, xps, yps, Ms, Ns, paths = [], [], [], [], [], []
    d0 = kind0 = None
    cu0 = None
    for X, Y in zip(Xs, Ys):
        k, xp, M, yp, N, d, kind, on_cuda, cu = _prep_pair(X, Y)
        if d0 is None:
            d0, kind0 = d, kind
        elif (d, kind) != (d0, kind0):
            raise ValueError("all pairs of a batch share dtype and feature dimension")
        cu0 = cu0 if cu0 is not None else cu
        keep.append(k)
        xps.append(xp)
        yps.append(yp)
        Ms.append(M)
        Ns.append(N)
        paths.append(_path_buffer(M, N, cu) if paths_out is None else paths_out[len(paths)])
    if cu0 is not None:
        _sync_stream(cu0)
    VP = ctypes.c_void_p * B
    I64 = ctypes.c_int64 * B
    K = I64()
    C = (ctypes.c_double * B)()
    rc = _get_lib().dtw_align_batch(B, VP(*xps), I64(*Ms), VP(*yps), I64(*Ns), d0,
                                    kind0 | _form(dp_f32, cost_bf16),
                             VP(*[p.data_ptr() for p in paths]), K, C)
    _check(rc, "dtw_align_batch")
    return [(paths[b][:K[b]], int(C[b]) if kind0 == ABS_I32 else C[b]) for b in range(B)]


def submit(X, Y, path_out=None, *, dp_f32: bool = False, cost_bf16: bool = False):
    """Queues one alignment; returns (ticket, path buffer, keep-alive)."""
    keep, xp, M, yp, N, d, kind, on_cuda, cu = _prep_pair(X, Y)
    if cu is not None:
        _sync_stream(cu)
    path = _path_buffer(M, N, cu) if path_out is None else path_out
    r = Request(xp, M, yp, N, d, kind | _form(dp_f32, cost_bf16), path.data_ptr())
    t = _check(_get_lib().dtw_submit(ctypes.byref(r)), "dtw_submit")
    return t, path, keep


def poll(ticket: int):
    """(status, K, D*) of a submitted request; status PENDING while it runs."""
    K, c = ctypes.c_int64(), ctypes.c_double()
    rc = _get_lib().dtw_poll(int(ticket), ctypes.byref(K), ctypes.byref(c))
    return rc, K.value, c.value


def wait(ticket: int, timeout_s: float = 120.0, interval_s: float = 2e-4):
    """Polls until the request is no longer pending; returns (status, K, D*)."""
    import time
    t_end = time.monotonic() + timeout_s
    while True:
        rc, K, c = poll(ticket)
        if rc != PENDING:
            return rc, K, c
        if time.monotonic() > t_end:
            raise TimeoutError(f"request {ticket} still pending after {timeout_s} s")
        time.sleep(interval_s)


def footprint(M: int, N: int, d: int = 1, kind: int = ABS_I32) -> int:
    return int(_get_lib().dtw_footprint(M, N, d, kind))


def set_budget(nbytes: int) -> None:
    _check(_get_lib().dtw_set_budget(int(nbytes)), "dtw_set_budget")


def set_arena(tensor_or_none) -> None:
    """Hands a CUDA tensor's storage to the library as its workspace (None releases it)."""
    if tensor_or_none is None:
        _check(_get_lib().dtw_set_arena(None, 0), "dtw_set_arena")
    else:
        t = tensor_or_none
        _check(_get_lib().dtw_set_arena(ctypes.c_void_p(t.data_ptr()), t.numel() * t.element_size()), "dtw_set_arena")


def set_option(key: int, value: int) -> None:
    _check(_get_lib().dtw_set_option(int(key), int(value)), "dtw_set_option")


def set_stream(stream) -> None:
    _get_lib().dtw_set_stream(ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream))


PIPE_OPS = ("min3_s32", "sad_u32", "ffma_f32", "ffma2_f32x2", "sqrt_rn_f32", "dadd_f64")
LATENCY_OPS = ("min3_s32", "sad_u32", "fadd_f32", "dadd_f64", "shfl_up")


def pipe_rates() -> dict:
    """Issue rates (thread instructions per second, whole device) of the
    instructions the per-cell roofline counts, measured on the current device."""
    out = (ctypes.c_double * len(PIPE_OPS))()
    n = _get_lib().dtw_pipe_rates(out, len(PIPE_OPS))
    if n < 0:
        raise DTWError(n, "dtw_pipe_rates")
    return {PIPE_OPS[i]: out[i] for i in range(n)}


def op_latencies() -> dict:
    """Dependent-chain latencies (cycles per operation, one warp) of the cell
    updates' chain operations, measured on the current device."""
    n_all = len(PIPE_OPS) + len(LATENCY_OPS)
    out = (ctypes.c_double * n_all)()
    n = _get_lib().dtw_pipe_rates(out, n_all)
    if n < 0:
        raise DTWError(n, "dtw_pipe_rates")
    return {LATENCY_OPS[i]: out[len(PIPE_OPS) + i] for i in range(max(0, n - len(PIPE_OPS)))}


def get_stats() -> dict:
    s = Stats()
    _check(_get_lib().dtw_get_stats(ctypes.byref(s)), "dtw_get_stats")
    return s.as_dict()
