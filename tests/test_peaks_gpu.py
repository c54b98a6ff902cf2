"""The pipe-rate probe (rt_pipe_peak) returns rates that the SM can physically issue: per
SM, at most 128 FP32 lanes per clock (the two lanes of FFMA2 counted) at the device's
highest SM clock, and MUFU functions at most at the FP32 rate."""

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    from paper_2509_03623_b300 import _rt, build
    assert torch.cuda.is_available()
    build.build()
    return _rt


def max_sm_hz():
    import torch
    return torch.cuda.get_device_properties(0).clock_rate * 1e3 if hasattr(
        torch.cuda.get_device_properties(0), "clock_rate") else 2.1e9


@pytest.mark.parametrize("op", ["ffma", "ffma2", "ex2", "rsqrt", "lg2", "rcp", "sqrt", "tanh",
                                "tanh_f16x2"])
def test_pipe_rates_are_physical(rt, op):
    r = rt.rt_pipe_peak(op, 4096)
    per_clk = r["per_s_sm"] / 2.2e9     # at or above any clock the SM reaches
    assert 2.0 <= per_clk <= 128.0 * 1.03 * (2.2e9 / 2.0e9), r
    assert r["ms"] > 0.0 and r["counter_mhz"] > 0.0


def test_mufu_slower_than_fma(rt):
    f = rt.rt_pipe_peak("ffma", 4096)["per_s_sm"]
    for op in ("ex2", "rsqrt", "lg2", "rcp", "sqrt"):
        assert rt.rt_pipe_peak(op, 4096)["per_s_sm"] < 0.6 * f, op
