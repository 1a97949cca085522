"""On-device microbenchmarks (pthr_measure_peak): each returns a positive
rate in the range a GB300 can deliver, and the pipes keep their documented
ratios (the packed f32x2 FMA issues at most as fast as the scalar FMA, the
integer-logic pipe at most as fast as the FMA pipe, FP64 far below FP32)."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import _lib  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402


@pytest.fixture(scope="module")
def rates():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    lib = _lib.load()
    scratch = torch.empty((4096 + (16 << 20),), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    out = {}
    for kind in range(6):
        r, t = ctypes.c_double(), ctypes.c_double()
        _lib.check(lib.pthr_measure_peak(kind, ctypes.c_void_p(scratch.data_ptr()), scratch.numel(),
                                         ctypes.c_void_p(st.cuda_stream), ctypes.byref(r), ctypes.byref(t)))
        assert t.value > 0
        out[kind] = r.value
    return out


def test_peak_rates_are_plausible(rates):
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    clk = 2.2e9                                   # above any GB300 SM clock
    assert 0.2 * n_sm * 128 * 1.0e9 < rates[_lib.PEAK_SMEM_READ] <= 1.05 * n_sm * 128 * clk
    assert 1e12 < rates[_lib.PEAK_L2_READ] < rates[_lib.PEAK_SMEM_READ]
    assert rates[_lib.PEAK_FMA] <= 1.05 * n_sm * 128 * clk
    assert rates[_lib.PEAK_ALU] <= 1.05 * rates[_lib.PEAK_FMA]
    assert rates[_lib.PEAK_FMA2] <= 1.05 * rates[_lib.PEAK_FMA]
    assert rates[_lib.PEAK_FP64] < 0.5 * rates[_lib.PEAK_FMA]
    print("PEAKS " + " ".join(f"{k}={v:.4g}" for k, v in rates.items()))
