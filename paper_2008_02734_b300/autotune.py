"""Autotuner of the sweep's lane block, the split windows and the base-case cutoff.

The integer sweep is compiled in four lane blocks (4, 2 or 8 rows per lane, 4
columns per step, and 4 rows with fully unrolled step groups:
DTW_OPT_SWEEP_VARIANT 0..3), each box of a level may be split on up to 1, 7 or
15 windows of split rows (DTW_OPT_SPLIT_WINDOWS), and the recursion hands boxes
to the full-table base case below a cutoff area (DTW_OPT_BASE_AREA).  None of
them changes a result -- the integer path is the canonical one at any cutoff
and split, and the lane block only reorders the same cell updates -- but all
change the time: a thinner band means more bands (more warps at the top levels,
a longer pipeline ramp), more windows fewer levels with longer sweeps, a larger
cutoff fewer, cheaper levels at the bottom.  ``tune`` times dtw_align on a
seeded synthetic pair of the caller's size for every candidate and applies the
fastest.
"""
from __future__ import annotations

import itertools

from . import OPT_BASE_AREA, OPT_SPLIT_WINDOWS, OPT_SWEEP_VARIANT, align, set_option
from . import synth

VARIANTS = (0, 1, 2, 3)
WINDOWS = (1, 7, 15)
BASE_AREAS = (4096, 16384, 32768)
# split windows tried for a batch: the integer batch takes 3, the d=12 chroma
# batch 15 (more of its work in the first level, whose sweeps keep every SM
# busy, and fewer of the deeper levels, which do not)
BATCH_WINDOWS = (1, 3, 7, 15)
# integer lane blocks tried for a batch: R=4 (variant 0) and R=8 (variant 2)
BATCH_INT_VARIANTS = (0, 2)
DEFAULT_WINDOWS = 7


def tune(M: int, N: int, *, variants=VARIANTS, windows=WINDOWS, base_areas=BASE_AREAS, reps: int = 3,
         apply: bool = True, flush_l2: bool = True) -> dict:
    """Times every (variant, windows, base area) on an integer pair of M x N
    frames with CUDA events (median of ``reps`` after one warm-up) and returns
    {"variant", "windows", "base_area", "ms", "table"}; with ``apply`` the
    fastest is set.  ``flush_l2``: each timed call starts with a cold L2 (a
    256 MiB write before it, outside the events), as in a stream of alignments
    of different pairs."""
    import torch

    X, Y = synth.int_pair(12345, M, N)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    path = torch.empty((M + N - 1, 2), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if flush_l2 else None
    table = []
    for v, w, a in itertools.product(variants, windows, base_areas):
        set_option(OPT_SWEEP_VARIANT, v)
        set_option(OPT_SPLIT_WINDOWS, w)
        set_option(OPT_BASE_AREA, a)
        align(Xd, Yd, path_out=path)
        ms = []
        for _ in range(reps):
            if flush is not None:
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            align(Xd, Yd, path_out=path)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        ms.sort()
        table.append({"variant": v, "windows": w, "base_area": a, "ms": ms[len(ms) // 2]})
    best = min(table, key=lambda r: r["ms"])
    set_option(OPT_SWEEP_VARIANT, best["variant"] if apply else 0)
    set_option(OPT_SPLIT_WINDOWS, best["windows"] if apply else DEFAULT_WINDOWS)
    set_option(OPT_BASE_AREA, best["base_area"] if apply else 16384)
    return {"variant": best["variant"], "windows": best["windows"], "base_area": best["base_area"], "ms": best["ms"],
            "table": table}


def tune_batch(Xs, Ys, *, base_areas=BASE_AREAS, windows=BATCH_WINDOWS, variants=None, reps: int = 2,
               apply: bool = True, **align_kw) -> dict:
    """The base-case cutoff, split windows and (integer data) lane block for a
    batch: times align_batch on the caller's own pairs (device tensors) for
    every candidate (median of ``reps`` after one warm-up) and returns
    {"variant", "base_area", "windows", "ms", "table"}; with ``apply`` the
    fastest is set.  ``variants`` defaults to BATCH_INT_VARIANTS for int32 data;
    float data has one lane block per dimension (variant None: left as it is).
    Results do not depend on any of them (integer paths are canonical; float
    paths are optimal within the float tolerance)."""
    import torch

    from . import align_batch

    if variants is None:
        variants = BATCH_INT_VARIANTS if Xs[0].dtype == torch.int32 else (None,)
    stream = torch.cuda.current_stream()
    table = []
    for v, w, a in itertools.product(variants, windows, base_areas):
        if v is not None:
            set_option(OPT_SWEEP_VARIANT, v)
        set_option(OPT_SPLIT_WINDOWS, w)
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
        table.append({"variant": v, "windows": w, "base_area": a, "ms": ms[len(ms) // 2]})
    best = min(table, key=lambda r: r["ms"])
    if best["variant"] is not None:
        set_option(OPT_SWEEP_VARIANT, best["variant"] if apply else 0)
    set_option(OPT_SPLIT_WINDOWS, best["windows"] if apply else DEFAULT_WINDOWS)
    set_option(OPT_BASE_AREA, best["base_area"] if apply else 16384)
    return {"variant": best["variant"], "base_area": best["base_area"], "windows": best["windows"], "ms": best["ms"],
            "table": table}
