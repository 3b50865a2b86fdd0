"""GPU parity of the mixed Neumann / Dirichlet wall pairs along x and y: the quarter-wave transforms
(DCT-IV, DST-IV) of the shared-memory line engine and of the warp-per-line kernels against scipy, and
the FP64 / mixed solves against the CPU oracle."""
import itertools

import numpy as np
import pytest
import scipy.fft

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD, ND, DN = 0, 1, 2, 3, 4
ALL = (P, NN, DD, ND, DN)
MIXED_XY = [c for c in itertools.product(ALL, ALL) if ND in c or DN in c]


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


def ref_forward(x, bc, axis):
    """Unnormalised forward transform in the library's slot order."""
    if bc == NN:
        return scipy.fft.dct(x, type=2, axis=axis)
    if bc == DD:
        return scipy.fft.dst(x, type=2, axis=axis)
    if bc == ND:
        return scipy.fft.dct(x, type=4, axis=axis)
    if bc == DN:
        return scipy.fft.dst(x, type=4, axis=axis)
    n = x.shape[axis]
    X = np.moveaxis(np.fft.rfft(x, axis=axis), axis, -1)
    out = np.empty(X.shape[:-1] + (n,))
    out[..., 0] = X[..., 0].real
    if n > 1:
        out[..., 1] = X[..., n // 2].real
    for k in range(1, n // 2):
        out[..., 2 * k] = X[..., k].real
        out[..., 2 * k + 1] = X[..., k].imag
    return np.moveaxis(out, -1, axis)


def make_plan(cans, n, bc, prec=0, sweeps=2, dzf=None, L=(1.0, 1.0)):
    o = cans.cans_opts_default()
    o.prec, o.max_sweeps = prec, sweeps
    return cans.cans_poisson_plan(n, L, bc, dzf, o)[1]


@pytest.mark.parametrize("bcx,bcy", MIXED_XY)
@pytest.mark.parametrize("n", [(16, 8, 3), (48, 96, 2), (2, 6, 2), (24, 18, 2), (1024, 32, 1)])
def test_quarter_wave_fp64_transforms(cans, bcx, bcy, n):
    h = make_plan(cans, n, (bcx, bcy, NN))
    x = np.random.default_rng(3).standard_normal((n[2], n[1], n[0]))
    t = dev(x)
    assert cans.cans_transform_xy(h, t.data_ptr(), 1, stream()) == 0
    want = ref_forward(ref_forward(x, bcx, 2), bcy, 1)
    got = host(t)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    assert cans.cans_transform_xy(h, t.data_ptr(), -1, stream()) == 0
    back = host(t)
    assert np.abs(back - n[0] * n[1] * x).max() <= 1e-13 * n[0] * n[1] * np.abs(x).max()
    cans.cans_plan_destroy(h)


@pytest.mark.parametrize("bcx,bcy", [(ND, P), (DN, NN), (P, ND), (NN, DN), (ND, DN), (DN, ND), (DD, ND)])
@pytest.mark.parametrize(
    "n", [(256, 512, 2), (512, 256, 1), (1024, 256, 1), (64, 48, 2), (24, 256, 2), (32, 1024, 2), (48, 256, 3)]
)
def test_quarter_wave_f32_transforms(cans, bcx, bcy, n):
    """The mixed path's float x / y passes: quarter-wave lines on the warp-per-line x kernels for N in
    {256, 512, 1024}, the lanes-across-x-slots y kernel for Ny in {256, 512, 1024} (Nx a multiple of
    16; several tiles and planes), the shared-memory engine otherwise."""
    import torch

    h = make_plan(cans, n, (bcx, bcy, NN), prec=1)
    x = np.random.default_rng(4).standard_normal((n[2], n[1], n[0]))
    t = dev(x)
    w = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    assert cans.cans_transform_xy_f32(h, t.data_ptr(), w.data_ptr(), 1, stream()) == 0
    want = ref_forward(ref_forward(x, bcx, 2), bcy, 1)
    got = host(w).astype(np.float64)
    assert np.abs(got - want).max() <= 4e-6 * np.abs(want).max()
    assert cans.cans_transform_xy_f32(h, t.data_ptr(), w.data_ptr(), -1, stream()) == 0
    back = host(t)
    assert np.abs(back - n[0] * n[1] * x).max() <= 4e-6 * n[0] * n[1] * np.abs(x).max()
    cans.cans_plan_destroy(h)


@pytest.mark.parametrize("bcx,bcy", MIXED_XY)
@pytest.mark.parametrize("bcz", [NN, DD, DN])
@pytest.mark.parametrize("prec", [0, 1])
def test_quarter_wave_solves_match_oracle(cans, bcx, bcy, bcz, prec):
    import torch

    n = (12, 18, 9)
    bc = (bcx, bcy, bcz)
    dzf = I.tanh_dzf(n[2], 1.8)
    f = I.uniform(111 + bcx + 5 * bcy + 25 * bcz, (n[2], n[1], n[0]), -1, 1)
    ref = oracle.poisson_solve(f, bc, (1.3, 0.9), dzf)
    s = cans.PoissonSolver(n, bc, (1.3, 0.9), dzf, prec=prec, sweeps=2)
    p = torch.empty_like(dev(f))
    _, info, st = s.solve(dev(f), p, info=True)
    s.close()
    assert st == 0, (st, info)
    got = host(p)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert err <= (1e-12 if prec == 0 else 1e-11), err


@pytest.mark.parametrize("n,bc", [((1, 8, 6), (ND, P, NN)), ((8, 1, 6), (P, DN, DD)), ((2, 2, 3), (ND, DN, NN)),
                                  ((256, 128, 16), (ND, P, NN)), ((128, 256, 16), (P, DN, NN))])
@pytest.mark.parametrize("prec", [0, 1])
def test_quarter_wave_edge_and_large_shapes(cans, n, bc, prec):
    """One-cell and two-cell directions, and warp-engine-sized shapes (quarter-wave lines on the
    warp-per-line kernels; the mixed residual in the fused warp x pass)."""
    import torch

    dzf = I.tanh_dzf(n[2], 1.5)
    f = I.uniform(131, (n[2], n[1], n[0]), -1, 1)
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=prec, sweeps=2)
    p = torch.empty_like(dev(f))
    _, info, st = s.solve(dev(f), p, info=True)
    s.close()
    assert st == 0, (st, info)
    res = oracle.relative_residual(host(p), f, bc, (1.0, 1.0), dzf, nthreads=8)
    assert res <= 1e-12, (res, info)
