"""Pins of the oracle's fractional step in a box whose directions are periodic or bounded by no-slip
walls (lid-driven cavity, square duct, channel, periodic Taylor-Green box), written separately from
the channel oracle.

Independent facts: with walls in z only it reproduces the separately written channel oracle (itself
pinned); projections leave discretely divergence-free fields and are idempotent; the advection
conserves kinetic energy on uniform grids (zero normal velocity at walls); a small-amplitude
Taylor-Green vortex in the periodic box decays by the RK3 polynomial of the closed-form discrete
eigenvalue 2 (4/h^2) sin^2(h/2); wall-bounded shear modes decay by the RK3 polynomial of their
closed-form no-slip eigenvalues; the cavity keeps the mirror symmetry of its lid-driven problem.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

CAVITY, DUCT, CHANNEL, PERIODIC = (1, 1, 1), (0, 1, 1), (0, 0, 1), (0, 0, 0)


def random_state(shape, walls, L, dzf, seed, amp=0.3):
    u = amp * I.uniform(seed, shape, -1, 1)
    v = amp * I.uniform(seed + 1, shape, -1, 1)
    w = amp * I.uniform(seed + 2, shape, -1, 1)
    for a, d in ((u, 2), (v, 1), (w, 0)):  # normal velocity on the high wall face is zero
        if walls[2 - d]:
            idx = [slice(None)] * 3
            idx[d] = -1
            a[tuple(idx)] = 0.0
    return oracle.box_project(u, v, w, walls, L, dzf)


def test_box_with_z_walls_is_the_channel():
    shape, L = (8, 6, 10), (2.0, 1.0)
    dzf = I.tanh_dzf(8, 1.8, 2.0)
    u, v, w = random_state(shape, CHANNEL, L, dzf, 5)
    u = u + 1.0
    p = 0.1 * I.uniform(9, shape, -1, 1)
    (au, av, aw), (lu, lv, lw) = oracle.box_operators(u, v, w, CHANNEL, L, dzf)
    ru, rv, rw = oracle.momentum_rhs(u, v, w, 0.03, L, dzf)
    for a, l, r in ((au, lu, ru), (av, lv, rv), (aw, lw, rw)):
        np.testing.assert_allclose(a + 0.03 * l, r, rtol=0, atol=1e-12 * np.abs(r).max())
    a = oracle.rk3_step(u, v, w, p, 0.03, 0.5, 1.0, L, dzf, dt=4e-3)
    b = oracle.box_rk3_step(u, v, w, p, CHANNEL, 0.03, L, dzf, ubulk=1.0, forcing=True, dt=4e-3)
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_allclose(y, x, rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))


@pytest.mark.parametrize("walls", [CAVITY, DUCT, CHANNEL, PERIODIC])
def test_box_projection_divergence_free_and_idempotent(walls):
    shape, L = (6, 8, 10), (1.0, 1.5)
    dzf = I.tanh_dzf(6, 1.5) if walls[2] else np.full(6, 1.0 / 6)
    u, v, w = random_state(shape, walls, L, dzf, 11)
    d = oracle.box_divergence(u, v, w, walls, L, dzf)
    assert np.abs(d).max() <= 1e-11
    u2, v2, w2 = oracle.box_project(u, v, w, walls, L, dzf)
    for a, b in ((u, u2), (v, v2), (w, w2)):
        assert np.abs(a - b).max() <= 1e-12


@pytest.mark.parametrize("walls", [CAVITY, DUCT, PERIODIC])
def test_box_advection_conserves_energy_on_uniform_grids(walls):
    shape, L = (8, 8, 8), (1.0, 1.0)
    dzf = np.full(8, 1.0 / 8)
    u, v, w = random_state(shape, walls, L, dzf, 21, amp=1.0)
    (au, av, aw), _ = oracle.box_operators(u, v, w, walls, L, dzf)
    work = float((u * au).sum() + (v * av).sum() + (w * aw).sum())
    scale = float(np.abs(u * au).sum() + np.abs(v * av).sum() + np.abs(w * aw).sum())
    assert abs(work) <= 1e-12 * scale, (work, scale)


def test_taylor_green_decays_by_the_rk3_polynomial():
    """u = U sin x cos y, v = -U cos x sin y on the staggered points of a periodic 2 pi box; with a tiny
    U the step is linear: u1 = R(-kappa dt) u0, R(z) = 1 + z + z^2/2 + z^3/6, kappa = 2 nu (4/h^2) sin^2(h/2)."""
    n = 16
    h = 2 * np.pi / n
    nz = 4
    xf, xc = (np.arange(n) + 1) * h, (np.arange(n) + 0.5) * h
    U = 1e-7
    u = U * np.sin(xf)[None, None, :] * np.cos(xc)[None, :, None] * np.ones((nz, 1, 1))
    v = -U * np.cos(xc)[None, None, :] * np.sin(xf)[None, :, None] * np.ones((nz, 1, 1))
    w = np.zeros_like(u)
    p = np.zeros_like(u)
    nu, dt = 0.2, 0.05
    dzf = np.full(nz, 1.0 / nz)
    un, vn, wn, pn, _ = oracle.box_rk3_step(u, v, w, p, PERIODIC, nu, (2 * np.pi, 2 * np.pi), dzf, dt=dt)
    z = -2 * nu * 4 / h ** 2 * np.sin(h / 2) ** 2 * dt
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6
    np.testing.assert_allclose(un, R * u, rtol=0, atol=1e-9 * U)
    np.testing.assert_allclose(vn, R * v, rtol=0, atol=1e-9 * U)
    assert np.abs(wn).max() <= 1e-12 * U


def test_lid_driven_cavity_keeps_its_mirror_symmetry():
    """A lid moving along x over a cavity started from rest: the problem is symmetric under y -> Ly - y
    (u, w even, v odd about the mid-plane); the step keeps the symmetry and is divergence-free."""
    shape, L = (8, 6, 10), (1.0, 1.0)
    dzf = I.tanh_dzf(8, 1.2)
    z = np.zeros(shape)
    u, v, w, p = z, z, z, z
    for _ in range(2):
        u, v, w, p, dt = oracle.box_rk3_step(u, v, w, p, CAVITY, 0.01, L, dzf, cfl=0.5, lid=1.0, dt=2e-3)
    assert u[-1].max() > 1e-3  # the lid has started to drag the top cells
    np.testing.assert_allclose(u, u[:, ::-1, :], rtol=0, atol=1e-12)
    np.testing.assert_allclose(w, w[:, ::-1, :], rtol=0, atol=1e-12)
    # v sits on y-faces: face j mirrors face ny - 2 - j, the wall face stays zero
    np.testing.assert_allclose(v[:, :-1, :], -v[:, -2::-1, :], rtol=0, atol=1e-12)
    assert np.all(v[:, -1, :] == 0.0) and np.all(u[:, :, -1] == 0.0) and np.all(w[-1] == 0.0)
    assert np.abs(oracle.box_divergence(u, v, w, CAVITY, L, dzf)).max() <= 1e-10


@pytest.mark.parametrize("comp,walls", [(0, (0, 1, 1)), (1, (1, 0, 1)), (2, (1, 1, 0))])
def test_wall_bounded_shear_mode_decays_by_the_rk3_polynomial(comp, walls):
    """One velocity component pointing along its own periodic direction and varying only across the
    two walled directions, as a product of the cell-centred no-slip eigenvectors sin(pi (a+1)(i+1/2)/N):
    advection-free and divergence-free, so one step multiplies it by R(nu lam dt), with
    lam = -sum over the walled directions of 4 sin^2(pi (a+1)/2N)/h^2 (catches a wrong wall ghost)."""
    n = (8, 6, 10)  # (nz, ny, nx)
    nz, ny, nx = n
    L = (1.0, 1.5)
    h = (L[0] / nx, L[1] / ny, 1.0 / nz)
    N = (nx, ny, nz)
    dzf = np.full(nz, h[2])
    modes = {0: 0, 1: 1, 2: 0}
    prof = np.ones(n)
    lam = 0.0
    for d in range(3):
        if d == comp or not walls[d]:
            continue
        a = modes[d]
        idx = np.arange(N[d])
        f = np.sin(np.pi * (a + 1) * (idx + 0.5) / N[d])
        shape = [1, 1, 1]
        shape[2 - d] = N[d]
        prof = prof * f.reshape(shape)
        lam -= 4 * np.sin(np.pi * (a + 1) / (2 * N[d])) ** 2 / h[d] ** 2
    fields = [np.zeros(n), np.zeros(n), np.zeros(n)]
    fields[comp] = prof.copy()
    p = np.zeros(n)
    nu, dt = 0.01, 2e-3
    out = oracle.box_rk3_step(*fields, p, walls, nu, L, dzf, dt=dt)
    z = nu * lam * dt
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6
    np.testing.assert_allclose(out[comp], R * prof, rtol=0, atol=1e-13)
    for c in range(3):
        if c != comp:
            assert np.abs(out[c]).max() <= 1e-13
