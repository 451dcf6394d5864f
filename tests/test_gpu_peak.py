"""The FMA-chain microbenchmark that measures the FP32 and FP64 rates the pair
sweeps are compared against."""
import pytest
import torch

from paper_2511_21921_gb300 import _lib as L

pytestmark = pytest.mark.gpu


def test_alu_peak_rates_are_plausible():
    st = torch.cuda.current_stream().cuda_stream
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32, ms32 = L.crk_alu_peak(st, False, 2048)
    f64, ms64 = L.crk_alu_peak(st, True, 64)
    assert ms32 > 0 and ms64 > 0
    # 128 FP32 lanes x 2 flops per SM per clock; clocks between 0.5 and 2.2 GHz
    assert sms * 128 * 2 * 0.5e9 < f32 < sms * 128 * 2 * 2.2e9
    assert 0 < f64 < f32


def test_alu_peak_argument_errors():
    st = torch.cuda.current_stream().cuda_stream
    for fp64, iters in ((False, 0), (True, -3)):
        with pytest.raises(L.CRKError):
            L.crk_alu_peak(st, fp64, iters)
    import ctypes as C
    f = C.c_double()
    assert L.load().crk_alu_peak(C.c_void_p(st), 2, 16, C.byref(f), None) == L.CRK_EINVAL
