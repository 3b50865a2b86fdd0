"""The mixed path's integer-arithmetic double/float conversions against IEEE round-to-nearest.

The nearest-float conversion must be bit-identical to the hardware (torch on the GPU) and to numpy
on the host for every input class: random bit patterns (zeros, subnormals, inf, NaN, every exponent),
values across the float range and its edges, and exact ties between two floats (ties to even).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def inputs():
    rng = np.random.default_rng(2024)
    bits = rng.integers(0, 2**63, size=200_000, dtype=np.int64).astype(np.uint64)
    bits[::2] |= np.uint64(1) << np.uint64(63)
    raw = bits.view(np.float64)
    exps = rng.integers(-160, 140, size=200_000)
    scaled = rng.uniform(-2, 2, size=exps.size) * np.exp2(exps.astype(np.float64))
    f32 = rng.standard_normal(100_000).astype(np.float32) * np.float32(3.0)
    nxt = np.nextafter(f32, np.float32(np.inf))
    ties = (f32.astype(np.float64) + nxt.astype(np.float64)) / 2  # exactly halfway between two floats
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, fmax, -fmax, fmax * (1 + 2**-25),
                      fmax * (1 + 2**-23), tiny, tiny / 2, tiny * (1 - 2**-30), 2.0**-149, 2.0**-150,
                      2.0**-151, 2.0**-80, 2.0**-81, 2.0**127, 2.0**128, 1 + 2**-24, 1 + 3 * 2**-24,
                      5e-324, 2.2250738585072014e-308, 1.7976931348623157e308])
    return np.concatenate([raw, scaled, ties, edges])


def test_nearest_float_and_split(cans):
    import torch

    x = inputs()
    n = x.size
    xd = torch.from_numpy(x).cuda()
    rn, hi, lo = (torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3))
    back = torch.empty(n, dtype=torch.float64, device="cuda")
    st = cans.cans_split_f64(xd.data_ptr(), n, rn.data_ptr(), hi.data_ptr(), lo.data_ptr(), back.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    assert st == 0
    hw = xd.float()
    torch.cuda.synchronize()
    rn_b = rn.cpu().numpy().view(np.uint32)
    # bit-identical to the hardware conversion for every input, NaN payloads included
    assert np.array_equal(rn_b, hw.cpu().numpy().view(np.uint32))
    # and to numpy's conversion for every non-NaN input
    ok = ~np.isnan(x)
    with np.errstate(over="ignore"):
        assert np.array_equal(rn_b[ok], x[ok].astype(np.float32).view(np.uint32))
    h, l, b = hi.cpu().numpy(), lo.cpu().numpy(), back.cpu().numpy()
    assert np.array_equal(h.view(np.uint32), rn_b)
    # hi + lo carries x to 2^-46 relative wherever both parts are normal floats
    sel = np.isfinite(x) & (np.abs(x) >= 2.0**-100) & (np.abs(x) < 2.0**127)
    err = np.abs((x[sel] - h[sel].astype(np.float64)) - l[sel].astype(np.float64))
    assert np.all(err <= 2.0**-46 * np.abs(x[sel]))
    # back = hi + lo in double: exact widening of both parts, one rounded add
    fin = np.isfinite(h) & np.isfinite(l)
    assert np.array_equal(b[fin], h[fin].astype(np.float64) + l[fin].astype(np.float64))


def test_empty_and_null_outputs(cans):
    import torch

    assert cans.cans_split_f64(0, 0) == 0
    x = torch.ones(5, dtype=torch.float64, device="cuda")
    rn = torch.zeros(5, dtype=torch.float32, device="cuda")
    assert cans.cans_split_f64(x.data_ptr(), 5, rn.data_ptr()) == 0
    torch.cuda.synchronize()
    assert torch.equal(rn, torch.ones(5, dtype=torch.float32, device="cuda"))
    assert cans.cans_split_f64(0, 5) != 0
