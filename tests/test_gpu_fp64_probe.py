"""The FP64 FMA probe (cans_fp64_fma_probe) whose rate bench.py uses as the denominator of the FP64
paths' fractions: a plausible rate, and argument checks."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def test_fp64_fma_probe_reports_a_plausible_rate(cans):
    """The FP64 FMA probe bench.py divides by: finite, positive, and below the FP32 issue rate's
    bound for one FP64 operation per lane per cycle (148 SMs x 128 lanes x 2 flops x 2.1 GHz)."""
    import ctypes

    import torch

    rate = cans.fp64_fma_tflops(iters=2000, reps=2)
    assert 0.05 < rate < 148 * 128 * 2 * 2.1e9 / 1e12, rate
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    fl = ctypes.c_size_t(0)
    assert cans.lib().cans_fp64_fma_probe(out.data_ptr(), 16, 10, None, ctypes.byref(fl)) == cans.CANS_ERR_ARG
