"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test ties the oracle to an independent fact: a library transform (scipy.fft), a library
eigen-solver or dense LU (numpy/scipy) applied to the stencil matrix, closed-form eigenpairs, a
manufactured solution, second-order convergence to a continuum solution, or a re-run in
__float128.  A plausible mistake (dropped term, wrong sign or index, transposed operand) fails at
least one of them; tests/test_oracle_mutations.py plants such mistakes to show it.
"""
import itertools

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

import oracle
from paper_2001_05234_b300 import inputs as I

P, NN, DD = oracle.BC_P, oracle.BC_NN, oracle.BC_DD
ALL_BC = (P, NN, DD)


def dense_operator(n, bc, length_xy, dzf):
    """Matrix of L_h assembled column by column from the oracle's stencil apply."""
    nx, ny, nz = n
    N = nx * ny * nz
    A = np.empty((N, N))
    e = np.zeros((nz, ny, nx))
    for c in range(N):
        e.flat[c] = 1.0
        A[:, c] = oracle.apply_laplacian(e, bc, length_xy, dzf, nthreads=1).ravel()
        e.flat[c] = 0.0
    return A


def is_singular(bc):
    return DD not in bc


def volumes(n, length_xy, dzf):
    nx, ny, nz = n
    return np.broadcast_to((dzf * length_xy[0] / nx * length_xy[1] / ny)[:, None, None], (nz, ny, nx)).ravel()


def dense_solve(A, f, w=None):
    """numpy dense LU; singular systems use the bordered matrix [[A, w], [w^T, 0]] (zero weighted mean)."""
    if w is None:
        return np.linalg.solve(A, f)
    N = A.shape[0]
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = A
    B[:N, N] = w
    B[N, :N] = w
    rhs = np.concatenate([f, [0.0]])
    return np.linalg.solve(B, rhs)[:N]


# ---------------------------------------------------------------------------------------------
# eigenbases
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc", ALL_BC)
@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 12, 17, 32])
def test_eigenbasis_orthonormal(bc, n):
    E, lam = oracle.eigenbasis(bc, n)
    assert np.abs(E.T @ E - np.eye(n)).max() < 1e-13


@pytest.mark.parametrize("bc", ALL_BC)
@pytest.mark.parametrize("n", [2, 3, 8, 12, 17, 24])
def test_eigenpairs_against_stencil(bc, n):
    """Closed-form eigenpairs satisfy the stencil matrix (unit spacing) and match numpy's eigvalsh."""
    A = dense_operator((n, 1, 1), (bc, P, NN), (float(n), 1.0), np.ones(1))
    E, lam = oracle.eigenbasis(bc, n)
    assert np.abs(A @ E - E * lam[None, :]).max() < 1e-12
    assert np.allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(lam), atol=1e-13, rtol=0)


@pytest.mark.parametrize("n", [4, 12, 33, 64])
def test_periodic_eigenvalues_match_cosine_form(n):
    """Periodic eigenvalue of wavenumber k equals 2(cos(2 pi k/n) - 1)."""
    _, lam = oracle.eigenbasis(P, n)
    k = (np.arange(n) + 1) // 2
    assert np.abs(lam - 2.0 * (np.cos(2 * np.pi * k / n) - 1.0)).max() < 1e-14


# ---------------------------------------------------------------------------------------------
# transforms: the oracle's basis against scipy.fft
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 5, 8, 16, 48, 100])
def test_neumann_basis_is_orthonormal_dct2(n):
    x = np.random.default_rng(n).standard_normal(n)
    E, _ = oracle.eigenbasis(NN, n)
    assert np.abs(E.T @ x - scipy.fft.dct(x, type=2, norm="ortho")).max() < 1e-13
    assert np.abs(E @ x - scipy.fft.dct(x, type=3, norm="ortho")).max() < 1e-13


@pytest.mark.parametrize("n", [2, 5, 8, 16, 48, 100])
def test_dirichlet_basis_is_orthonormal_dst2(n):
    x = np.random.default_rng(n + 1).standard_normal(n)
    E, _ = oracle.eigenbasis(DD, n)
    assert np.abs(E.T @ x - scipy.fft.dst(x, type=2, norm="ortho")).max() < 1e-13
    assert np.abs(E @ x - scipy.fft.dst(x, type=3, norm="ortho")).max() < 1e-13


@pytest.mark.parametrize("n", [2, 3, 8, 9, 16, 48, 64])
def test_periodic_basis_is_real_dft(n):
    x = np.random.default_rng(n + 2).standard_normal(n)
    E, _ = oracle.eigenbasis(P, n)
    X = np.fft.rfft(x)
    want = np.empty(n)
    want[0] = X[0].real / np.sqrt(n)
    kmax = n // 2 - 1 if n % 2 == 0 else (n - 1) // 2
    for k in range(1, kmax + 1):
        want[2 * k - 1] = np.sqrt(2.0 / n) * X[k].real
        want[2 * k] = -np.sqrt(2.0 / n) * X[k].imag
    if n % 2 == 0:
        want[n - 1] = X[n // 2].real / np.sqrt(n)
    assert np.abs(E.T @ x - want).max() < 1e-13


# ---------------------------------------------------------------------------------------------
# z rows and Thomas
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bcz", [NN, DD])
def test_z_rows_match_stencil(bcz):
    dzf = I.tanh_dzf(11, 1.8, 2.0)
    a, b, c = oracle.z_rows(bcz, dzf)
    A = dense_operator((1, 1, 11), (P, P, bcz), (1.0, 1.0), dzf)
    T = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    assert np.abs(A - T).max() < 1e-9 * np.abs(A).max()


def test_thomas_against_solve_banded():
    rng = np.random.default_rng(3)
    n = 57
    a, c = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    b = -(a + c) - rng.uniform(0.01, 1, n)
    a[0] = 0.0
    c[-1] = 0.0
    d = rng.standard_normal(n)
    ab = np.zeros((3, n))
    ab[0, 1:] = c[:-1]
    ab[1] = b
    ab[2, :-1] = a[1:]
    assert np.abs(oracle.thomas(a, b, c, d) - scipy.linalg.solve_banded((1, 1), ab, d)).max() < 1e-12


def test_pure_z_problem_reduces_to_banded_solve():
    """nx = ny = 1 periodic: the 3-D solve is one tridiagonal solve along the stretched z grid."""
    dzf = I.tanh_dzf(40, 2.0, 1.0)
    f = np.random.default_rng(4).standard_normal((40, 1, 1))
    p = oracle.poisson_solve(f, (P, P, DD), dzf=dzf)
    A = dense_operator((1, 1, 40), (P, P, DD), (1.0, 1.0), dzf)
    ab = np.zeros((3, 40))
    ab[0, 1:] = np.diag(A, 1)
    ab[1] = np.diag(A)
    ab[2, :-1] = np.diag(A, -1)
    ref = scipy.linalg.solve_banded((1, 1), ab, f.ravel())
    assert np.abs(p.ravel() - ref).max() < 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------------------------------------
# brute force: dense LU on small grids, every boundary-condition combination
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc", list(itertools.product(ALL_BC, ALL_BC, ALL_BC)))
def test_dense_lu_8cubed(bc):
    n = (8, 8, 8)
    dzf = I.uniform_dzf(8) if bc[2] == P else I.tanh_dzf(8, 1.8)
    L = (1.0, 1.3)
    rng = np.random.default_rng(sum(bc) + 10 * bc[0] + 3 * bc[1])
    f = rng.uniform(-1, 1, (8, 8, 8))
    w = volumes(n, L, dzf) if is_singular(bc) else None
    if w is not None:
        f = f - (f.ravel() @ w) / w.sum()
    A = dense_operator(n, bc, L, dzf)
    ref = dense_solve(A, f.ravel(), w).reshape(f.shape)
    p = oracle.poisson_solve(f, bc, L, dzf)
    assert np.linalg.norm(p - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("bc", [(P, DD, NN), (NN, NN, NN), (DD, P, DD), (P, P, P)])
def test_dense_lu_ragged(bc):
    n = (6, 5, 7)
    dzf = I.uniform_dzf(7, 1.5) if bc[2] == P else I.tanh_dzf(7, 1.2, 1.5)
    L = (2.0, 0.7)
    f = np.random.default_rng(5).uniform(-1, 1, (7, 5, 6))
    w = volumes(n, L, dzf) if is_singular(bc) else None
    if w is not None:
        f = f - (f.ravel() @ w) / w.sum()
    ref = dense_solve(dense_operator(n, bc, L, dzf), f.ravel(), w).reshape(f.shape)
    p = oracle.poisson_solve(f, bc, L, dzf)
    assert np.linalg.norm(p - ref) / np.linalg.norm(ref) < 1e-12


# ---------------------------------------------------------------------------------------------
# manufactured solutions
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [(P, P, NN), (P, DD, NN), (NN, DD, DD), (DD, NN, NN)])
def test_manufactured_discrete_solution(bc):
    n = (24, 16, 20)
    dzf = I.tanh_dzf(20, 1.8)
    L = (2.0, 1.0)
    p0 = np.random.default_rng(6).standard_normal((20, 16, 24))
    if is_singular(bc):
        p0 = I.weighted_mean_removed(p0, dzf)
    f = oracle.apply_laplacian(p0, bc, L, dzf)
    p = oracle.poisson_solve(f, bc, L, dzf)
    assert np.linalg.norm(p - p0) / np.linalg.norm(p0) < 1e-12


def _continuum_error(m):
    """x periodic, y Dirichlet, z Neumann, uniform unit cube: p = cos(2 pi x) sin(pi y) cos(pi z)."""
    n = (m, m, m)
    h = 1.0 / m
    c = (np.arange(m) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    pe = np.cos(2 * np.pi * x) * np.sin(np.pi * y) * np.cos(np.pi * z)
    f = -(4 * np.pi ** 2 + np.pi ** 2 + np.pi ** 2) * pe
    p = oracle.poisson_solve(f, (P, DD, NN), (1.0, 1.0), I.uniform_dzf(m))
    return np.abs(p - pe).max()


def test_second_order_convergence_to_continuum():
    e = [_continuum_error(m) for m in (8, 16, 32)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.7 < r1 < 4.3 and 3.85 < r2 < 4.15, e


def test_second_order_on_stretched_z():
    errs = []
    for m in (16, 32, 64):
        dzf = I.tanh_dzf(m, 1.5)
        zc = I.z_centres(dzf)
        c = (np.arange(8) + 0.5) / 8
        pe = np.cos(np.pi * zc)[:, None, None] * np.ones((1, 1, 8))
        f = -(np.pi ** 2) * pe
        p = oracle.poisson_solve(f, (P, P, NN), (1.0, 1.0), dzf)
        p = p - (p[:, 0, 0] * dzf).sum() + (pe[:, 0, 0] * dzf).sum()
        errs.append(np.abs(p - pe).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


# ---------------------------------------------------------------------------------------------
# exact result within round-off: __float128 and long double re-runs of the same source
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [(P, P, NN), (P, DD, NN), (NN, NN, DD)])
def test_fp64_matches_quad_precision(bc):
    n = (12, 10, 16)
    dzf = I.tanh_dzf(16, 1.8)
    f = np.random.default_rng(7).uniform(-1, 1, (16, 10, 12))
    if is_singular(bc):
        f = I.weighted_mean_removed(f, dzf)
    p64 = oracle.poisson_solve(f, bc, (1.0, 1.0), dzf, prec=64)
    p80 = oracle.poisson_solve(f, bc, (1.0, 1.0), dzf, prec=80)
    p128 = oracle.poisson_solve(f, bc, (1.0, 1.0), dzf, prec=128)
    nrm = np.linalg.norm(p128)
    assert np.linalg.norm(p64 - p128) / nrm < 1e-13
    assert np.linalg.norm(p80 - p128) / nrm < 1e-16


# ---------------------------------------------------------------------------------------------
# invariants on the 32^3 workload
# ---------------------------------------------------------------------------------------------
def test_uniform32_residual_and_gauge():
    case = I.case_uniform32()
    f = I.rhs_host(case)
    p = oracle.poisson_solve(f, case.bc, case.length_xy, case.dzf)
    assert oracle.relative_residual(p, f, case.bc, case.length_xy, case.dzf) <= 1e-13
    w = volumes(case.n, case.length_xy, case.dzf)
    assert abs(p.ravel() @ w) / (np.abs(p).ravel() @ w) < 1e-14


def test_rk3_coefficients_golden():
    rows = np.loadtxt(__file__.replace("test_oracle_pins.py", "golden/rk3_coefficients.txt"))
    alpha = rows[:, 1] / rows[:, 2]
    beta = rows[:, 3] / rows[:, 4]
    gamma = alpha + beta
    assert abs(gamma.sum() - 1.0) < 1e-15  # three substages advance one full step
    assert np.allclose(gamma, [8 / 15, 2 / 15, 1 / 3])
