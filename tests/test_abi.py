"""The C-ABI library builds, loads and exports every function include/dtw_b300.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dtw_b300.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2008_02734_b300 import build
    build.build()
    import paper_2008_02734_b300 as dtw
    return dtw


def declared_functions():
    src = open(HEADER).read()
    return re.findall(r"^DTW_API\s+[\w\s\*]+?\b(dtw_\w+)\s*\(", src, flags=re.M)


def test_header_declares_abi():
    names = declared_functions()
    assert len(names) >= 12
    assert {"dtw_align", "dtw_cost", "dtw_align_batch", "dtw_submit", "dtw_poll"} <= set(names)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib.LIB_PATH], text=True)
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib.lib, name)
    assert set(lib.ABI_FUNCTIONS) == set(declared_functions())


def test_header_compiles_as_c(tmp_path):
    c = tmp_path / "t.c"
    c.write_text('#include "dtw_b300.h"\nint main(void){ dtw_stats s; (void)s; return DTW_OK; }\n')
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           "-c", str(c), "-o", str(tmp_path / "t.o")])


def test_strerror_and_options(lib):
    assert lib.lib.dtw_strerror(0) == b"ok"
    assert lib.lib.dtw_strerror(-4) == b"device-side wait timed out"
    assert lib.lib.dtw_set_option(999, 1) == lib.EINVAL
    assert lib.lib.dtw_set_option(lib.OPT_BASE_AREA, 2) == lib.EINVAL
    assert lib.lib.dtw_set_option(lib.OPT_BASE_AREA, 1 << 20) == lib.EINVAL
    for bad in (0, 16, -1):
        assert lib.lib.dtw_set_option(lib.OPT_SPLIT_WINDOWS, bad) == lib.EINVAL
    assert lib.lib.dtw_set_option(lib.OPT_SPLIT_WINDOWS, 7) == 0


def test_pipe_rates_checks_arguments_on_host(lib):
    out = (ctypes.c_double * 6)()
    assert lib.lib.dtw_pipe_rates(None, 6) == lib.EINVAL
    assert lib.lib.dtw_pipe_rates(out, 0) == lib.EINVAL


def test_invalid_arguments_rejected_on_host(lib):
    X = np.zeros(4, np.int32)
    p = np.zeros(16, np.int32)
    c = ctypes.c_double()
    L = lib.lib
    # M < 1, d mismatch, unknown kind, null pointers: all rejected before any CUDA call
    assert L.dtw_align(X.ctypes.data, 0, X.ctypes.data, 4, 1, 1, p.ctypes.data, ctypes.byref(c)) == lib.EINVAL
    assert L.dtw_align(X.ctypes.data, 4, X.ctypes.data, 4, 2, 1, p.ctypes.data, ctypes.byref(c)) == lib.EINVAL
    assert L.dtw_align(X.ctypes.data, 4, X.ctypes.data, 4, 1, 7, p.ctypes.data, ctypes.byref(c)) == lib.EINVAL
    assert L.dtw_align(None, 4, X.ctypes.data, 4, 1, 1, p.ctypes.data, ctypes.byref(c)) == lib.EINVAL
    assert L.dtw_align(X.ctypes.data, 4, X.ctypes.data, 4, 1, 1, None, ctypes.byref(c)) == lib.EINVAL
    assert L.dtw_cost(X.ctypes.data, 4, X.ctypes.data, 4, 1, 1 | lib.PLAIN_F64, ctypes.byref(c)) == lib.EINVAL
    assert L.dtw_align_batch(0, None, None, None, None, 1, 1, None, None, None) == lib.EINVAL
    assert L.dtw_poll(123456, None, None) == lib.EINVAL


def test_footprint_is_linear(lib):
    f1 = lib.footprint(10000, 12000)
    f2 = lib.footprint(20000, 24000)
    f4 = lib.footprint(40000, 48000)
    assert 1.8 < f2 / f1 < 2.2 and 1.8 < f4 / f2 < 2.2
    # well under the M*N*4 bytes = 1.9 GB of a full table (the split rows of up to
    # seven windows per box are the largest part)
    assert f2 < 128 << 20
    assert lib.footprint(0, 5) == 0
