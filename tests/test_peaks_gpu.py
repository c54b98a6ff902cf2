"""The pipe-rate probe (rt_pipe_peak) returns rates that the SM can physically issue: at
most 128 FP32 lanes per clock per SM for FFMA (256 counting the two lanes of FFMA2), at most
the FP32 rate for the MUFU functions, and a clock implied by cycles / wall time within the
device's range."""

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    from paper_2509_03623_b300 import _rt, build
    assert torch.cuda.is_available()
    build.build()
    return _rt


@pytest.mark.parametrize("op,lo,hi", [("ffma", 64, 132), ("ffma2", 64, 264), ("ex2", 8, 132),
                                       ("rsqrt", 4, 132), ("lg2", 4, 132), ("rcp", 4, 132),
                                       ("sqrt", 4, 132), ("tanh", 4, 132),
                                       ("tanh_f16x2", 4, 264)])
def test_pipe_rates_are_physical(rt, op, lo, hi):
    r = rt.rt_pipe_peak(op, 2048)
    assert lo <= r["per_clk_sm"] <= hi, r
    assert 300.0 <= r["sm_mhz"] <= 2300.0, r
    assert r["ms"] > 0.0
