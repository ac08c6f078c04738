"""dtw_pipe_rates: the instruction rates the per-cell roofline is set against
come out positive and in the order the pipes' widths fix (a fused multiply-add
pipe outruns the FP64 adder and the multi-instruction square root)."""
import pytest

import paper_2008_02734_b300 as dtw


@pytest.mark.gpu
def test_pipe_rates_plausible():
    r = dtw.pipe_rates()
    assert set(r) == set(dtw.PIPE_OPS)
    assert all(v > 0 for v in r.values())
    # at least one SM's worth of lanes per nanosecond for the wide pipes
    for k in ("min3_s32", "sad_u32", "ffma_f32", "ffma2_f32x2"):
        assert r[k] > 1e11, (k, r[k])
    assert r["ffma_f32"] > 4 * r["dadd_f64"]
    assert r["ffma_f32"] > r["sqrt_rn_f32"]


@pytest.mark.gpu
def test_op_latencies_plausible():
    """The dependent-chain latencies: positive, a shuffle and an FP64 add slower
    than the one-instruction integer minimum on the chain."""
    lat = dtw.op_latencies()
    assert set(lat) == set(dtw.LATENCY_OPS)
    assert all(1.0 < v < 10000.0 for v in lat.values()), lat
    assert lat["dadd_f64"] > lat["fadd_f32"]
    assert lat["shfl_up"] > lat["min3_s32"]
