"""GPU parity of the Helmholtz form (L_h + sigma) p = f (Eq. up_id_2) and of the interior z-face
grid of a staggered w, through the C ABI, against the CPU oracle."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD = 0, 1, 2


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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(cans, f_full, n, bc, L, dzf, prec, shift, z_grid=0, sweeps=2, per_call=False):
    """Solve on the GPU; f_full has the caller's (Nz, Ny, Nx) shape.  Returns (p, info, status)."""
    import torch

    s = cans.PoissonSolver(n, bc, L, dzf, prec=prec, sweeps=sweeps, shift=0.0 if per_call else shift,
                           z_grid=z_grid)
    f = dev(f_full)
    p = torch.full_like(f, 7.0)  # the face grid must leave the top plane alone
    _, info, st = s.solve(f, p, info=True, shift=shift if per_call else None)
    out = host(p)
    s.close()
    return out, info, st


@pytest.mark.parametrize("bcx,bcy", list(itertools.product((P, NN, DD), (P, NN, DD))))
@pytest.mark.parametrize("bcz", [NN, DD])
@pytest.mark.parametrize("prec", [0, 1])
def test_shifted_solve_all_boundary_conditions(cans, bcx, bcy, bcz, prec):
    n = (24, 18, 17)
    bc = (bcx, bcy, bcz)
    dzf = I.tanh_dzf(n[2], 1.8)
    f = I.uniform(31 + bcx + 3 * bcy + 9 * bcz, (n[2], n[1], n[0]), -1, 1)
    shift = -40.0
    ref = oracle.helmholtz_solve(f, bc, (1.2, 0.8), dzf, shift=shift)
    got, info, st = run(cans, f, n, bc, (1.2, 0.8), dzf, prec, shift)
    assert st == 0, (st, info)
    assert rel(got, ref) <= (1e-12 if prec == 0 else 1e-11), rel(got, ref)
    res = oracle.relative_residual(got, f, bc, (1.2, 0.8), dzf, shift=shift)
    assert res <= 1e-12, res


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shift", [-1.0, -2.5e5])
def test_warp_engine_sizes_shifted(cans, prec, shift):
    """Shapes that take the warp-per-line x and y kernels and the streaming residual stencil; a small
    shift and an implicit-diffusion-sized one (-2 / (gamma nu dt))."""
    n = (256, 256, 24)
    bc = (P, P, NN)
    dzf = I.tanh_dzf(n[2], 1.8)
    f = I.uniform(41, (n[2], n[1], n[0]), -1, 1)
    got, info, st = run(cans, f, n, bc, (1.0, 1.0), dzf, prec, shift, sweeps=2)
    assert st == 0, (st, info)
    res = oracle.relative_residual(got, f, bc, (1.0, 1.0), dzf, shift=shift, nthreads=8)
    assert res <= 1e-12, (res, info)


@pytest.mark.parametrize("bcx,bcy", [(P, P), (P, DD), (NN, NN), (DD, NN)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shift", [0.0, -60.0])
def test_face_grid_matches_oracle(cans, bcx, bcy, prec, shift):
    """z_grid 1: unknowns on the Nz - 1 interior faces of tanh cells, w = 0 on the walls; the top plane of
    the caller's arrays is neither read nor written."""
    ncell = 19
    n = (24, 16, ncell)
    bc = (bcx, bcy, DD)
    dzf = I.tanh_dzf(ncell, 1.8)
    f = I.uniform(51 + bcx + 3 * bcy, (ncell, n[1], n[0]), -1, 1)
    f[-1] = np.nan  # the wall plane must not be read
    ref = oracle.helmholtz_solve(f[:-1], bc, (1.0, 1.5), dzf, shift=shift, z_grid=1)
    got, info, st = run(cans, f, n, bc, (1.0, 1.5), dzf, prec, shift, z_grid=1)
    assert st == 0, (st, info)
    assert np.all(got[-1] == 7.0)
    assert rel(got[:-1], ref) <= (1e-12 if prec == 0 else 1e-11), rel(got[:-1], ref)


def test_face_grid_warp_engine_mixed(cans):
    ncell = 33
    n = (256, 128, ncell)
    bc = (P, P, DD)
    dzf = I.tanh_dzf(ncell, 1.8)
    f = I.uniform(61, (ncell, n[1], n[0]), -1, 1)
    got, info, st = run(cans, f, n, bc, (2.0, 1.0), dzf, 1, -3.0e3, z_grid=1, sweeps=2)
    assert st == 0, (st, info)
    res = oracle.relative_residual(got[:-1], f[:-1], bc, (2.0, 1.0), dzf, shift=-3.0e3, z_grid=1, nthreads=8)
    assert res <= 1e-12, (res, info)


@pytest.mark.parametrize("prec", [0, 1])
def test_per_call_shift_on_a_singular_plan(cans, prec):
    """cans_helmholtz_solve with a shift on a plan whose own problem is singular (x, y periodic, z
    Neumann): no gauge is applied during the call, and the plan's Poisson solve afterwards is the
    zero-mean singular solution again."""
    import torch

    n = (32, 24, 16)
    bc = (P, P, NN)
    dzf = I.tanh_dzf(n[2], 1.8)
    f = I.uniform(71, (n[2], n[1], n[0]), -1, 1)
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=prec, sweeps=2)
    fd = dev(f)
    p = torch.empty_like(fd)
    s.solve(fd, p, shift=-5.0)
    ref = oracle.helmholtz_solve(f, bc, (1.0, 1.0), dzf, shift=-5.0)
    assert rel(host(p), ref) <= 1e-11
    fc = I.weighted_mean_removed(f, dzf)
    s.solve(dev(fc), p)
    ref0 = oracle.poisson_solve(fc, bc, (1.0, 1.0), dzf)
    assert rel(host(p), ref0) <= 1e-11
    s.close()


def test_shift_argument_checks(cans):
    import torch

    s = cans.PoissonSolver((8, 8, 8), (P, P, DD), prec=0)
    f = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    st = cans.cans_helmholtz_solve(s.plan, f.data_ptr(), f.data_ptr(), 1.0, 0, 0)
    assert st == cans.CANS_ERR_ARG
    st = cans.cans_helmholtz_solve(s.plan, f.data_ptr(), f.data_ptr(), float("nan"), 0, 0)
    assert st == cans.CANS_ERR_ARG
    s.close()


@pytest.mark.parametrize("z_grid", [0, 1])
def test_adjoint_with_shift(cans, z_grid):
    """<S f, g> = <f, S^T g> for the shifted operator (the similarity S^T = D S D^-1 holds with the
    shift, D the control-volume widths of the grid solved)."""
    import torch

    ncell = 14
    n = (16, 12, ncell)
    bc = (P, NN, DD)
    dzf = I.tanh_dzf(ncell, 1.8)
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=0, shift=-9.0, z_grid=z_grid)
    nu = ncell - z_grid
    f = dev(I.uniform(81, (ncell, n[1], n[0]), -1, 1))
    g = dev(I.uniform(82, (ncell, n[1], n[0]), -1, 1))
    if z_grid:
        f[-1] = 0.0
        g[-1] = 0.0
    Sf = s.solve(f)
    STg = s.solve_adjoint(g)
    a = float((Sf[:nu] * g[:nu]).sum())
    b = float((f[:nu] * STg[:nu]).sum())
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b)), (a, b)
    s.close()


ND, DN = 3, 4


@pytest.mark.parametrize("bcz", [ND, DN])
@pytest.mark.parametrize("bcx,bcy", [(P, P), (NN, DD), (DD, NN), (P, NN)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shift", [0.0, -30.0])
def test_mixed_z_walls_match_oracle(cans, bcz, bcx, bcy, prec, shift):
    """Neumann at one z wall and Dirichlet at the other (the z rows, the residual stencils' ghosts and
    the FP64 norms take each wall's own rule); never singular."""
    n = (24, 18, 21)
    bc = (bcx, bcy, bcz)
    dzf = I.tanh_dzf(n[2], 1.8)
    f = I.uniform(91 + bcx + 3 * bcy + 9 * bcz, (n[2], n[1], n[0]), -1, 1)
    ref = oracle.helmholtz_solve(f, bc, (1.0, 1.0), dzf, shift=shift)
    got, info, st = run(cans, f, n, bc, (1.0, 1.0), dzf, prec, shift)
    assert st == 0, (st, info)
    assert rel(got, ref) <= (1e-12 if prec == 0 else 1e-11), rel(got, ref)
    res = oracle.relative_residual(got, f, bc, (1.0, 1.0), dzf, shift=shift)
    assert res <= 1e-12, res
    if prec == 0:
        assert abs(info[0] - res) <= 1e-3 * res + 1e-16  # the library's own FP64 norm of the same residual


@pytest.mark.parametrize("bcz", [ND, DN])
def test_mixed_z_walls_warp_engine_and_streaming_residual(cans, bcz):
    n = (256, 256, 40)
    bc = (P, P, bcz)
    dzf = I.tanh_dzf(n[2], 1.8)
    f = I.uniform(101 + bcz, (n[2], n[1], n[0]), -1, 1)
    got, info, st = run(cans, f, n, bc, (1.0, 1.0), dzf, 1, 0.0, sweeps=2)
    assert st == 0, (st, info)
    res = oracle.relative_residual(got, f, bc, (1.0, 1.0), dzf, nthreads=8)
    assert res <= 1e-12, (res, info)
