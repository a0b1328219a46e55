"""The ALU peak probe the benchmark reports beside the kick's roofline:
measured rates must sit below the device's nominal peaks (152 SMs x 128
FP32 lanes x 2 x 2070 MHz = 80.5 TFLOP/s; FP64 at 1/64 of that) and within a
factor of a few of them, and the FP64 rate far below the FP32 one."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_gives_plausible_peaks():
    from paper_2601_19654_gb300.build import build
    build()
    from paper_2601_19654_gb300 import opal
    p = opal.probe_alu_peaks()
    assert 20.0 < p["fp32_tflops"] <= 81.0, p
    assert 0.3 < p["fp64_tflops"] <= 2.6, p
    assert p["fp64_tflops"] < p["fp32_tflops"] / 16, p
    assert 0.5 < p["mufu_rsqrt_tops"] < 40.0, p
