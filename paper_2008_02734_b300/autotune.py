"""Autotuner of the sweep's lane block and of the base-case cutoff.

The integer sweep is compiled in three lane blocks (4, 2 or 8 rows per lane, 4
columns per step: DTW_OPT_SWEEP_VARIANT 0, 1, 2) and the recursion hands boxes to
the full-table base case below a cutoff area (DTW_OPT_BASE_AREA).  Neither
changes a result -- the integer path is the canonical one at any cutoff, and the
lane block only reorders the same cell updates -- but both change the time: a
thinner band means more bands (more warps at the top levels, a longer pipeline
ramp), a larger cutoff means fewer, cheaper levels at the bottom.  ``tune`` times
dtw_align on a seeded synthetic pair of the caller's size for every candidate
and applies the fastest.
"""
from __future__ import annotations

import itertools

from . import OPT_BASE_AREA, OPT_SWEEP_VARIANT, align, set_option
from . import synth

VARIANTS = (0, 1, 2, 3)
BASE_AREAS = (4096, 16384, 32768)


def tune(M: int, N: int, *, variants=VARIANTS, base_areas=BASE_AREAS, reps: int = 3, apply: bool = True) -> dict:
    """Times every (variant, base area) on an integer pair of M x N frames with
    CUDA events (median of ``reps`` after one warm-up) and returns
    {"variant", "base_area", "ms", "table"}; with ``apply`` the fastest is set."""
    import torch

    X, Y = synth.int_pair(12345, M, N)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    path = torch.empty((M + N - 1, 2), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    table = []
    for v, a in itertools.product(variants, base_areas):
        set_option(OPT_SWEEP_VARIANT, v)
        set_option(OPT_BASE_AREA, a)
        align(Xd, Yd, path_out=path)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            align(Xd, Yd, path_out=path)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        ms.sort()
        table.append({"variant": v, "base_area": a, "ms": ms[len(ms) // 2]})
    best = min(table, key=lambda r: r["ms"])
    set_option(OPT_SWEEP_VARIANT, best["variant"] if apply else 0)
    set_option(OPT_BASE_AREA, best["base_area"] if apply else 16384)
    return {"variant": best["variant"], "base_area": best["base_area"], "ms": best["ms"], "table": table}


def tune_batch(Xs, Ys, *, base_areas=BASE_AREAS, reps: int = 2, apply: bool = True, **align_kw) -> dict:
    """The base-case cutoff for a batch: times align_batch on the caller's own
    pairs (device tensors) for every candidate area (median of ``reps`` after
    one warm-up) and returns {"base_area", "ms", "table"}; with ``apply`` the
    fastest is set.  Results do not depend on the cutoff (integer paths are
    canonical; float paths are optimal within the float tolerance)."""
    import torch

    from . import align_batch

    stream = torch.cuda.current_stream()
    table = []
    for a in base_areas:
        set_option(OPT_BASE_AREA, a)
        align_batch(Xs, Ys, **align_kw)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            align_batch(Xs, Ys, **align_kw)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        ms.sort()
        table.append({"base_area": a, "ms": ms[len(ms) // 2]})
    best = min(table, key=lambda r: r["ms"])
    set_option(OPT_BASE_AREA, best["base_area"] if apply else 16384)
    return {"base_area": best["base_area"], "ms": best["ms"], "table": table}
