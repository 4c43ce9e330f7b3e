"""fabf_pipe_peaks, the measured denominators of the rooflines: every figure
is positive and finite, the SM clock read from clock64 against the global
timer is a plausible GPU clock, and the pipes keep their order on GB300
(FP32 FMA far above FP64 FMA; MUFU below the FP32 FMA rate)."""
import math

import pytest

torch = pytest.importorskip("torch")

from paper_1811_02308_gb300 import build, fabf  # noqa: E402

pytestmark = pytest.mark.gpu


def test_pipe_peaks_are_measured_and_ordered():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    p = fabf.fabf_pipe_peaks(0)
    for k in ("fp64_tflops", "fp32_tflops", "int32_tops", "mufu_tops", "sm_mhz"):
        assert math.isfinite(p[k]) and p[k] > 0, (k, p[k])
    assert p["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 300.0 <= p["sm_mhz"] <= 3500.0
    assert p["fp32_tflops"] > 10 * p["fp64_tflops"]
    assert p["mufu_tops"] < p["fp32_tflops"] / 2
    # no more than the FP32 FMA units can do at the measured clock (2 flops
    # per FMA, 128 lanes per SM), with 5 % slack for the clock's sampling
    bound = 2 * 128 * p["sms"] * p["sm_mhz"] * 1e6 / 1e12
    assert p["fp32_tflops"] <= 1.05 * bound
