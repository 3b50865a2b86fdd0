"""Pins of the oracle's RK3 step with Crank-Nicolson diffusion (Eq. up_id, Eq. up_id_2, the projection
and the pressure update with -gamma nu dt/2 L Phi).

Independent facts: a wall-parallel shear mode of the cell grid (advection-free, divergence-free)
decays by the closed-form product over the three substages of (1 + h lam)/(1 - h lam),
h = gamma_k nu dt / 2, lam its discrete eigenvalue; with a vanishing viscosity the step reduces to the
explicit RK3 step (pinned separately); without forcing the step converges at second order in time;
the new velocity is discretely divergence-free.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

GAMMA = (8 / 15, 5 / 12 - 17 / 60, 3 / 4 - 5 / 12)


@pytest.mark.parametrize("m", [0, 2])
def test_shear_mode_decays_by_the_crank_nicolson_factors(m):
    nx, ny, nz = 6, 4, 12
    h = 2.0 / nz
    dzf = np.full(nz, h)
    k = np.arange(nz)
    mode_u = np.sin(np.pi * (m + 1) * (k + 0.5) / nz)
    mode_v = np.sin(np.pi * (m + 2) * (k + 0.5) / nz)
    u = np.broadcast_to(mode_u[:, None, None], (nz, ny, nx)).copy()
    v = 0.5 * np.broadcast_to(mode_v[:, None, None], (nz, ny, nx)).copy()
    w = np.zeros_like(u)
    p = np.zeros_like(u)
    nu, dt = 0.05, 0.02
    un, vn, wn, pn, _ = oracle.rk3_step_implicit(u, v, w, p, nu, 0.5, 0.0, (1.0, 1.0), dzf, dt=dt, forcing=False)

    def factor(mm):
        lam = -4 * np.sin(np.pi * (mm + 1) / (2 * nz)) ** 2 / h ** 2
        out = 1.0
        for g in GAMMA:
            hh = g * nu * dt / 2
            out *= (1 + hh * lam) / (1 - hh * lam)
        return out

    np.testing.assert_allclose(un, factor(m) * u, rtol=0, atol=1e-13)
    np.testing.assert_allclose(vn, factor(m + 1) * v, rtol=0, atol=1e-13)
    assert np.abs(wn).max() <= 1e-13 and np.abs(pn).max() <= 1e-11


def _state(n, seed, amp=0.2):
    nx, ny, nz = n
    dzf = I.tanh_dzf(nz, 1.8) * 2.0
    zc = np.cumsum(dzf) - dzf / 2
    base = 1.5 * zc * (2 - zc)
    u = base[:, None, None] + amp * I.uniform(seed, (nz, ny, nx), -1, 1)
    v = amp * I.uniform(seed + 1, (nz, ny, nx), -1, 1)
    w = amp * I.uniform(seed + 2, (nz, ny, nx), -1, 1)
    w[-1] = 0.0
    u, v, w = oracle.project(u, v, w, (2.0, 1.0), dzf)[:3]
    p = 0.1 * I.uniform(seed + 3, (nz, ny, nx), -1, 1)
    return u, v, w, p, dzf


def test_vanishing_viscosity_reduces_to_the_explicit_step():
    n = (8, 6, 10)
    u, v, w, p, dzf = _state(n, 100)
    a = oracle.rk3_step(u, v, w, p, 1e-13, 0.5, 1.0, (2.0, 1.0), dzf, dt=0.01)
    b = oracle.rk3_step_implicit(u, v, w, p, 1e-13, 0.5, 1.0, (2.0, 1.0), dzf, dt=0.01)
    for x, y in zip(a[:4], b[:4]):
        assert np.abs(x - y).max() <= 1e-10 * max(1.0, np.abs(x).max())


def test_implicit_step_is_second_order_in_time():
    """Without the bulk forcing the Crank-Nicolson RK3 step converges at second order in time (the
    per-substage forcing shift makes both the explicit and the implicit step first order)."""
    u0, v0, w0, p0, dzf = _state((8, 6, 10), 200, amp=0.1)
    T = 0.016

    def integrate(dt):
        u, v, w, p = u0, v0, w0, p0
        for _ in range(int(round(T / dt))):
            u, v, w, p, _ = oracle.rk3_step_implicit(u, v, w, p, 0.02, 0.5, 1.0, (2.0, 1.0), dzf, dt=dt, forcing=False)
        return u, v, w

    ref = integrate(T / 128)
    errs = []
    for m in (2, 4, 8):
        r = integrate(T / m)
        errs.append(max(np.abs(r[i] - ref[i]).max() for i in range(3)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.6) and np.all(ratios < 4.6), (errs, ratios)


def test_implicit_step_is_divergence_free():
    n = (8, 6, 10)
    u, v, w, p, dzf = _state(n, 300)
    un, vn, wn, pn, dt = oracle.rk3_step_implicit(u, v, w, p, 0.01, 0.5, 1.0, (2.0, 1.0), dzf, dt=5e-3)
    d = oracle.divergence(un, vn, wn, (2.0, 1.0), dzf)
    assert np.abs(d).max() <= 1e-10
    assert np.all(wn[-1] == 0.0)
