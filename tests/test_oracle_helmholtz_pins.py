"""Pins of the oracle's Helmholtz form (L_h + sigma) p = f (Eq. up_id_2, the implicit-diffusion step
solved "with the same type of direct solver" as the pressure) and of its face grid for a staggered
w (unknowns on the interior z-faces, w = 0 on the wall faces), and of the mixed Neumann / Dirichlet
wall pairs along z.

Independent facts used: closed-form discrete eigenpairs (periodic cosines, the cell-centred
Neumann / Dirichlet cosines and sines, and the node-Dirichlet sines of the face grid, whose
eigenvalues are -4 sin^2(pi m / 2N) / h^2, and the quarter-wave cosines / sines of a mixed wall
pair), numpy dense LU of the operator assembled from the
stencil, the oracle's separate channel w-diffusion (the viscous part of the momentum right-hand
side), and a re-run in __float128.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

P, NN, DD = oracle.BC_P, oracle.BC_NN, oracle.BC_DD


def dense_helmholtz(shape, bc, length_xy, dzf, shift, z_grid):
    nz, ny, nx = shape
    N = nx * ny * nz
    A = np.empty((N, N))
    e = np.zeros(shape)
    for c in range(N):
        e.flat[c] = 1.0
        A[:, c] = oracle.apply_helmholtz(e, bc, length_xy, dzf, shift=shift, z_grid=z_grid, nthreads=1).ravel()
        e.flat[c] = 0.0
    return A


@pytest.mark.parametrize("shift", [-0.5, -37.0, -4.0e4])
def test_shifted_eigenfunction_cell_grid(shift):
    """f = an eigenvector of the x (periodic), y (Neumann) and z (Dirichlet, uniform) operators:
    the solution is f / (lam + shift) with the closed-form eigenvalues."""
    nx, ny, nz = 12, 10, 8
    lx, ly = 1.3, 0.7
    dx, dy, h = lx / nx, ly / ny, 1.0 / nz
    a, b, m = 2, 3, 4
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    fx = np.cos(2 * np.pi * a * i / nx)
    fy = np.cos(np.pi * b * (j + 0.5) / ny)
    fz = np.sin(np.pi * (m + 1) * (k + 0.5) / nz)
    f = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    lam = (-4 * np.sin(np.pi * a / nx) ** 2 / dx ** 2 - 4 * np.sin(np.pi * b / (2 * ny)) ** 2 / dy ** 2
           - 4 * np.sin(np.pi * (m + 1) / (2 * nz)) ** 2 / h ** 2)
    p = oracle.helmholtz_solve(f, (P, NN, DD), (lx, ly), np.full(nz, h), shift=shift)
    np.testing.assert_allclose(p, f / (lam + shift), rtol=0, atol=1e-13 * np.abs(f / (lam + shift)).max())


@pytest.mark.parametrize("m", [1, 3, 6])
@pytest.mark.parametrize("shift", [0.0, -25.0])
def test_face_grid_node_dirichlet_eigenfunction(m, shift):
    """Face grid of a uniform z with Nz cells: the Nz - 1 interior faces are the interior nodes of a
    node-Dirichlet problem, eigenvectors sin(pi m (k+1) / Nz), eigenvalues -4 sin^2(pi m / 2Nz) / h^2."""
    nx, ny, nz = 8, 6, 9
    dx, dy, h = 1.0 / nx, 1.0 / ny, 1.0 / nz
    a = 1
    i, k = np.arange(nx), np.arange(nz - 1)
    fx = np.cos(2 * np.pi * a * i / nx)
    fz = np.sin(np.pi * m * (k + 1) / nz)
    f = np.broadcast_to(fz[:, None, None] * fx[None, None, :], (nz - 1, ny, nx)).copy()
    lam = -4 * np.sin(np.pi * a / nx) ** 2 / dx ** 2 - 4 * np.sin(np.pi * m / (2 * nz)) ** 2 / h ** 2
    p = oracle.helmholtz_solve(f, (P, P, DD), (1.0, 1.0), np.full(nz, h), shift=shift, z_grid=1)
    ref = f / (lam + shift)
    np.testing.assert_allclose(p, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("bc", [(P, P, NN), (NN, DD, NN), (DD, P, DD), (NN, NN, NN)])
@pytest.mark.parametrize("shift", [-1.0, -300.0])
def test_dense_lu_helmholtz_cell_grid(bc, shift):
    shape = (5, 4, 6)
    dzf = I.uniform(5, (shape[0],), 0.5, 1.5)
    f = I.uniform(9, shape, -1, 1)
    A = dense_helmholtz(shape, bc, (1.1, 0.9), dzf, shift, 0)
    ref = np.linalg.solve(A, f.ravel()).reshape(shape)
    got = oracle.helmholtz_solve(f, bc, (1.1, 0.9), dzf, shift=shift)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("bxy", list(itertools.product((P, NN, DD), (P, NN, DD))))
def test_dense_lu_face_grid(bxy):
    ncell = 7
    dzf = I.uniform(6, (ncell,), 0.5, 1.5)
    shape = (ncell - 1, 4, 6)
    f = I.uniform(10, shape, -1, 1)
    bc = (bxy[0], bxy[1], DD)
    A = dense_helmholtz(shape, bc, (1.0, 1.2), dzf, -3.0, 1)
    ref = np.linalg.solve(A, f.ravel()).reshape(shape)
    got = oracle.helmholtz_solve(f, bc, (1.0, 1.2), dzf, shift=-3.0, z_grid=1)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_face_grid_operator_is_the_channel_w_diffusion():
    """The face-grid operator equals the viscous part of the oracle's own channel momentum right-hand
    side for w (rhs(nu = 1) - rhs(nu = 0), u = v = 0), a routine written separately for the RK3 step."""
    nx, ny, ncell = 6, 5, 8
    dzf = I.tanh_dzf(ncell, 1.8) * 2.0
    shape = (ncell, ny, nx)
    w = I.uniform(12, shape, -1, 1)
    w[-1] = 0.0  # the top wall face
    z = np.zeros(shape)
    L = (1.7, 0.9)
    r1 = oracle.momentum_rhs(z, z, w, 1.0, L, dzf)[2]
    r0 = oracle.momentum_rhs(z, z, w, 0.0, L, dzf)[2]
    lap = oracle.apply_helmholtz(w[:-1], (P, P, DD), L, dzf, shift=0.0, z_grid=1)
    np.testing.assert_allclose((r1 - r0)[:-1], lap, rtol=0, atol=1e-10 * np.abs(lap).max())


@pytest.mark.parametrize("z_grid", [0, 1])
def test_helmholtz_fp64_matches_quad(z_grid):
    ncell = 10
    dzf = I.tanh_dzf(ncell, 1.8)
    shape = (ncell - z_grid, 6, 8)
    f = I.uniform(13, shape, -1, 1)
    bc = (P, NN, DD)
    a = oracle.helmholtz_solve(f, bc, (1.0, 1.0), dzf, shift=-7.0, z_grid=z_grid, prec=64)
    b = oracle.helmholtz_solve(f, bc, (1.0, 1.0), dzf, shift=-7.0, z_grid=z_grid, prec=128)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


def test_zero_shift_is_the_poisson_solve():
    dzf = I.tanh_dzf(8, 1.8)
    f = I.weighted_mean_removed(I.uniform(14, (8, 6, 4), -1, 1), dzf)
    a = oracle.helmholtz_solve(f, (P, P, NN), (1.0, 1.0), dzf, shift=0.0)
    b = oracle.poisson_solve(f, (P, P, NN), (1.0, 1.0), dzf)
    np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------------------------------------
# mixed walls along z: Neumann at the low wall and Dirichlet at the high wall (ND), or the reverse
# ---------------------------------------------------------------------------------------------
ND, DN = oracle.BC_ND, oracle.BC_DN


@pytest.mark.parametrize("bcz", [ND, DN])
@pytest.mark.parametrize("m", [0, 3])
def test_mixed_wall_quarter_wave_eigenfunction(bcz, m):
    """Uniform z with a Neumann and a Dirichlet wall: the eigenvectors are the quarter-wave cosines
    cos(pi (m + 1/2)(k + 1/2) / N) (ND) or sines sin(...) (DN), eigenvalues -4 sin^2(pi (2m+1) / 4N) / h^2."""
    nx, ny, nz = 6, 4, 10
    h = 1.0 / nz
    k = np.arange(nz)
    th = np.pi * (m + 0.5) * (k + 0.5) / nz
    fz = np.cos(th) if bcz == ND else np.sin(th)
    fx = np.cos(2 * np.pi * np.arange(nx) / nx)
    f = fz[:, None, None] * np.ones((1, ny, 1)) * fx[None, None, :]
    lam = -4 * np.sin(np.pi / nx) ** 2 * nx ** 2 - 4 * np.sin(np.pi * (2 * m + 1) / (4 * nz)) ** 2 / h ** 2
    p = oracle.poisson_solve(f, (P, P, bcz), (1.0, 1.0), np.full(nz, h))
    np.testing.assert_allclose(p, f / lam, rtol=0, atol=1e-13 * np.abs(f / lam).max())


@pytest.mark.parametrize("bcz", [ND, DN])
@pytest.mark.parametrize("bxy", [(P, P), (NN, NN), (P, DD), (NN, P)])
def test_dense_lu_mixed_walls(bcz, bxy):
    shape = (6, 4, 5)
    dzf = I.uniform(15, (shape[0],), 0.5, 1.5)
    f = I.uniform(16, shape, -1, 1)
    bc = (bxy[0], bxy[1], bcz)
    A = dense_helmholtz(shape, bc, (1.0, 1.3), dzf, 0.0, 0)
    ref = np.linalg.solve(A, f.ravel()).reshape(shape)  # a Dirichlet wall: never singular
    got = oracle.poisson_solve(f, bc, (1.0, 1.3), dzf)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_mixed_walls_are_the_two_ends_of_nn_and_dd():
    """Row by row, the ND rows are the NN rows near the low wall and the DD rows near the high wall."""
    dzf = I.uniform(17, (9,), 0.5, 1.5)
    nn, dd, nd, dn = (oracle.z_rows(b, dzf) for b in (NN, DD, ND, DN))
    for q in range(3):
        np.testing.assert_array_equal(nd[q][:4], nn[q][:4])
        np.testing.assert_array_equal(nd[q][-4:], dd[q][-4:])
        np.testing.assert_array_equal(dn[q][:4], dd[q][:4])
        np.testing.assert_array_equal(dn[q][-4:], nn[q][-4:])


@pytest.mark.parametrize("bc", [ND, DN])
@pytest.mark.parametrize("n", [1, 2, 5, 8, 12])
def test_quarter_wave_basis_is_the_dct4_dst4(bc, n):
    """The oracle's x / y basis for a mixed wall pair: orthonormal, E^T x equal to scipy's DCT-IV
    (ND) / DST-IV (DN) up to its factor 2 sqrt(n/2), and eigenpairs of the 1-D stencil matrix with a
    mirrored (Neumann) ghost at one end and a negated (Dirichlet) ghost at the other."""
    import scipy.fft

    E, lam = oracle.eigenbasis(bc, n)
    np.testing.assert_allclose(E.T @ E, np.eye(n), atol=1e-13)
    x = I.uniform(18 + n, (n,), -1, 1)
    t = scipy.fft.dct(x, type=4) if bc == ND else scipy.fft.dst(x, type=4)
    np.testing.assert_allclose(E.T @ x, t / 2 * np.sqrt(2.0 / n), atol=1e-13)
    T = np.diag(np.full(n, -2.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    lo, hi = (1.0, -1.0) if bc == ND else (-1.0, 1.0)
    T[0, 0] += lo
    T[-1, -1] += hi
    np.testing.assert_allclose(T @ E, E * lam[None, :], atol=1e-12)


@pytest.mark.parametrize("bx,by", [(ND, P), (DN, NN), (P, ND), (ND, DN), (DN, DD)])
@pytest.mark.parametrize("bz", [NN, DD, ND])
def test_dense_lu_mixed_walls_in_x_and_y(bx, by, bz):
    shape = (4, 5, 6)
    dzf = I.uniform(19, (shape[0],), 0.5, 1.5)
    f = I.uniform(20, shape, -1, 1)
    bc = (bx, by, bz)
    A = dense_helmholtz(shape, bc, (1.2, 0.8), dzf, 0.0, 0)
    ref = np.linalg.solve(A, f.ravel()).reshape(shape)
    got = oracle.poisson_solve(f, bc, (1.2, 0.8), dzf)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
