"""Pins of the oracle's fractional-step pieces (divergence, gradient, momentum right-hand side,
stable time step, projection, RK3 step) against facts other than themselves."""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

SHAPE = (8, 6, 10)  # (nz, ny, nx)
L = (1.0, 0.7)


def rand_face(seed, shape=SHAPE):
    rng = np.random.default_rng(seed)
    u, v, w = (rng.standard_normal(shape) for _ in range(3))
    w[-1] = 0.0  # top wall face
    return u, v, w


def face_weights(dzf, shape=SHAPE):
    """Face volumes (x, y spacing common factor dropped): u, v faces dzf_k, w faces dzc_{k+1/2}."""
    nz = shape[0]
    dzc = np.empty(nz)
    dzc[:-1] = 0.5 * (dzf[:-1] + dzf[1:])
    dzc[-1] = dzf[-1]
    wu = np.broadcast_to(dzf[:, None, None], shape)
    ww = np.broadcast_to(dzc[:, None, None], shape).copy()
    ww[-1] = 0.0  # the wall face carries no unknown
    return wu, ww


@pytest.mark.parametrize("stretched", [False, True])
def test_divergence_is_minus_adjoint_of_gradient(stretched):
    """<D u, q>_cells = -<u, G q>_faces with cell and face volumes (summation by parts)."""
    dzf = I.tanh_dzf(SHAPE[0], 1.6, 2.0) if stretched else I.uniform_dzf(SHAPE[0], 2.0)
    u, v, w = rand_face(1)
    q = np.random.default_rng(2).standard_normal(SHAPE)
    d = oracle.divergence(u, v, w, L, dzf)
    gx, gy, gz = oracle.gradient(q, L, dzf)
    wu, ww = face_weights(dzf)
    lhs = float((d * q * dzf[:, None, None]).sum())
    rhs = -float((u * gx * wu).sum() + (v * gy * wu).sum() + (w * gz * ww).sum())
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_divergence_of_gradient_is_the_poisson_operator():
    """D G equals L_h of Eq. poi with periodic x, y and Neumann z (pins both against the Poisson oracle)."""
    dzf = I.tanh_dzf(SHAPE[0], 1.6, 2.0)
    q = np.random.default_rng(3).standard_normal(SHAPE)
    gx, gy, gz = oracle.gradient(q, L, dzf)
    dg = oracle.divergence(gx, gy, gz, L, dzf)
    lq = oracle.apply_laplacian(q, (0, 0, 1), L, dzf)
    assert np.abs(dg - lq).max() < 1e-11 * np.abs(lq).max()


def test_projection_is_divergence_free_idempotent_and_self_adjoint():
    dzf = I.tanh_dzf(SHAPE[0], 1.6, 2.0)
    u, v, w = rand_face(4)
    pu, pv, pw, _ = oracle.project(u, v, w, L, dzf)
    assert np.abs(oracle.divergence(pu, pv, pw, L, dzf)).max() < 1e-11
    assert np.abs(pw[-1]).max() == 0.0
    ppu, ppv, ppw, _ = oracle.project(pu, pv, pw, L, dzf)
    assert max(np.abs(ppu - pu).max(), np.abs(ppv - pv).max(), np.abs(ppw - pw).max()) < 1e-11
    # W_f-weighted self-adjointness: <P a, b>_W = <a, P b>_W
    a, b = rand_face(5), rand_face(6)
    Pa, Pb = oracle.project(*a, L, dzf)[:3], oracle.project(*b, L, dzf)[:3]
    wu, ww = face_weights(dzf)
    ip = lambda x, y: float((x[0] * y[0] * wu).sum() + (x[1] * y[1] * wu).sum() + (x[2] * y[2] * ww).sum())
    assert abs(ip(Pa, b) - ip(a, Pb)) < 1e-11 * abs(ip(Pa, b))


def test_advection_conserves_kinetic_energy_on_uniform_grid():
    """Conservative central advection of a divergence-free field does no work: <u, A(u)> = 0."""
    dzf = I.uniform_dzf(SHAPE[0], 2.0)
    u, v, w = oracle.project(*rand_face(7), L, dzf)[:3]
    ru, rv, rw = oracle.momentum_rhs(u, v, w, 0.0, L, dzf)
    wu, ww = face_weights(dzf)
    work = float((u * ru * wu).sum() + (v * rv * wu).sum() + (w * rw * ww).sum())
    scale = float(np.abs(u * ru * wu).sum())
    assert abs(work) < 1e-12 * scale


def test_diffusion_of_shear_profile_matches_stencil():
    """u = u(z) only: no advection; nu L u is the 1-D no-slip (Dirichlet-ghost) z operator."""
    dzf = I.tanh_dzf(SHAPE[0], 1.6, 2.0)
    prof = np.random.default_rng(8).standard_normal(SHAPE[0])
    u = np.broadcast_to(prof[:, None, None], SHAPE).copy()
    z = np.zeros(SHAPE)
    ru, rv, rw = oracle.momentum_rhs(u, z, z, 0.3, L, dzf)
    a, b, c = oracle.z_rows(2, dzf)
    want = 0.3 * (b * prof + np.concatenate([[0], a[1:] * prof[:-1]]) + np.concatenate([c[:-1] * prof[1:], [0]]))
    assert np.abs(ru[:, 0, 0] - want).max() < 1e-12 * np.abs(want).max()
    assert np.abs(rv).max() == 0 and np.abs(rw).max() == 0


def test_stable_dt_closed_form():
    """Uniform streamwise flow U: the largest inverse time scale is U / dx, so dt = cfl sqrt(3) dx / U."""
    dzf = I.uniform_dzf(SHAPE[0], 2.0)
    u = np.full(SHAPE, 2.0)
    z = np.zeros(SHAPE)
    dx = L[0] / SHAPE[2]
    assert abs(oracle.stable_dt(u, z, z, 1e-6, 0.9, L, dzf) - 0.9 * np.sqrt(3) * dx / 2.0) < 1e-14
    # viscous limit: dt = cfl * 1.65 dl^2 / nu with dl the smallest spacing
    dl = min(dx, L[1] / SHAPE[1], dzf.min())
    assert abs(oracle.stable_dt(u * 1e-9, z, z, 10.0, 0.9, L, dzf) - 0.9 * 1.65 * dl * dl / 10.0) < 1e-15


def test_rk3_step_keeps_flow_divergence_free_and_bulk_velocity():
    dzf = I.tanh_dzf(SHAPE[0], 1.6, 2.0)
    zc = I.z_centres(dzf)
    u, v, w = rand_face(9)
    u = 0.1 * u + 1.5 * (1 - (zc[:, None, None] - 1) ** 2)
    v, w = 0.1 * v, 0.1 * w
    u, v, w = oracle.project(u, v, w, L, dzf)[:3]
    p = np.zeros(SHAPE)
    u1, v1, w1, p1, dt = oracle.rk3_step(u, v, w, p, 2 / 5600, 0.9, 1.0, L, dzf)
    assert dt > 0
    assert np.abs(oracle.divergence(u1, v1, w1, L, dzf)).max() < 1e-10
    wsum = (dzf[:, None, None] * u1).sum() / (dzf.sum() * SHAPE[1] * SHAPE[2])
    assert abs(wsum - 1.0) < 1e-13


def test_rk3_third_order_on_linear_decay():
    """The low-storage RK3 of the paper is third order in time.

    v = eps cos(2 pi x) is divergence free (no pressure correction) and, with a tiny amplitude, only
    diffuses (advection is second order in eps); on this linear problem the differences between
    runs with dt, dt/2, dt/4 over a fixed interval shrink by ~2^3."""
    shape = (4, 4, 16)
    dzf = I.uniform_dzf(4, 1.0)
    Lxy = (1.0, 1.0)
    x = (np.arange(16) + 0.5) / 16  # v sits at cell centres in x
    v0 = 1e-6 * np.broadcast_to(np.cos(2 * np.pi * x)[None, None, :], shape).copy()
    nu = 0.05
    T = 0.4
    runs = []
    for nsteps in (8, 16, 32):
        dt = T / nsteps
        u, v, w, p = np.zeros(shape), v0.copy(), np.zeros(shape), np.zeros(shape)
        for _ in range(nsteps):
            u, v, w, p, _ = oracle.rk3_step(u, v, w, p, nu, 0.9, 0.0, Lxy, dzf, dt=dt)
        runs.append(v)
    d1 = np.abs(runs[0] - runs[1]).max()
    d2 = np.abs(runs[1] - runs[2]).max()
    assert 7.0 < d1 / d2 < 9.0, (d1, d2)
