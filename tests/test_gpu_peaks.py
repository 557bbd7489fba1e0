"""The arithmetic-peak microbenchmarks (cfft_measure_peak) that the roofline fractions
divide by: each returns a finite rate inside the bounds the hardware's unit counts set
(FP32: 128 lanes x 2 flops per SM per clock at most at 2070 MHz), the bf16 tensor rate
agrees with the cuBLAS bf16 GEMM the measured-peaks record holds, and kind::tf32 runs at
about half the bf16 rate (half the K per instruction at the same shape).  Nothing here
waits without a bound: the tensor kernels' mbarrier waits give up and report."""
import json
import os

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_measured_peaks_are_plausible(torch_cuda):
    from paper_1404_7357_gb300 import cfft
    sms = torch_cuda.cuda.get_device_properties(0).multi_processor_count
    fp32, ms32 = cfft.measure_peak(0, cfft.PEAK_FP32, reps=3)
    fp64, ms64 = cfft.measure_peak(0, cfft.PEAK_FP64, reps=3)
    tf32, mst = cfft.measure_peak(0, cfft.PEAK_TF32, reps=3)
    bf16, msb = cfft.measure_peak(0, cfft.PEAK_BF16, reps=3)
    print("SMs %d: FP32 %.1f TFLOP/s (%.2f ms), FP64 %.2f (%.2f ms), TF32 tensor %.0f (%.2f ms), "
          "BF16 tensor %.0f (%.2f ms)" % (sms, fp32, ms32, fp64, ms64, tf32, mst, bf16, msb))
    fp32_bound = sms * 128 * 2 * 2070e6 / 1e12
    assert 0.3 * fp32_bound < fp32 < 1.02 * fp32_bound
    assert 0.0 < fp64 < fp32
    assert 0.35 < tf32 / bf16 < 0.65
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            ref = json.load(f).get("bf16_tflops")
        if ref:
            assert 0.7 * ref < bf16 < 1.3 * ref
