"""The measured roofline denominators (shared-memory load bandwidth, packed
FP32 FMA throughput): positive, below the units' nominal ceilings with some
slack for clock boosts, and not far below them."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_plausible():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2207_00233_gb300 import build
    build.build()
    import paper_2207_00233_gb300 as fse
    smem, fp32 = fse.fse_measure_peaks(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # 128 B/clk and 128 FP32 lanes per SM at <= 2.2 GHz
    smem_ceiling = sms * 128 * 2.2e9 / 1e9
    fp32_ceiling = sms * 128 * 2 * 2.2e9 / 1e12
    print("smem GB/s", smem, "fp32 TFLOP/s", fp32)
    assert 0.3 * smem_ceiling < smem <= smem_ceiling
    assert 0.3 * fp32_ceiling < fp32 <= fp32_ceiling


def test_measure_peaks_rejects_bad_arguments():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import ctypes
    import paper_2207_00233_gb300 as fse
    L = fse.lib()
    assert L.fse_measure_peaks(0, None, None) == 1
    a, b = ctypes.c_double(), ctypes.c_double()
    assert L.fse_measure_peaks(-1, ctypes.byref(a), ctypes.byref(b)) == 1
