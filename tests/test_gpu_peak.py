"""The measured FP32 FMA throughput (the FFT path's roofline denominator):
positive, and not above the nominal rate of the device's FP32 lanes at the
maximum SM clock (152 SMs x 128 lanes x 2 flop x 2.07 GHz on a GB300), with a
small margin for the clock reading."""

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fp32_fma_peak_is_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04298_gb300 import fwr
    fwr.load()
    tflops, ms = fwr.fp32_fma_peak()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2 * 2.07e9 / 1e12
    print("FP32 FMA: %.1f TFLOP/s measured, %.1f nominal (%.3f ms per launch)" % (tflops, nominal, ms))
    assert 0.5 * nominal < tflops < 1.05 * nominal
    assert ms > 0
