"""The measured FP32 multiply-add ceiling (fmbym_fp32_fma_rate) that the benchmark divides by."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_fp32_fma_rate_is_near_the_alu_count():
    from paper_2203_00459_gb300 import build
    build.build()
    from paper_2203_00459_gb300 import _lib
    from paper_2203_00459_gb300.search import fp32_fma_rate
    rate = fp32_fma_rate(iters=20000, reps=2)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # 128 FP32 lanes per SM; the SM clock lies between a few hundred MHz and about 2.1 GHz
    assert 0.25 * sms * 128 * 1.0e9 < rate < sms * 128 * 2.2e9, rate
    import ctypes
    v = ctypes.c_double()
    assert _lib.lib().fmbym_fp32_fma_rate(None, 0, 1, ctypes.byref(v)) == _lib.ERR_INVALID_ARG
