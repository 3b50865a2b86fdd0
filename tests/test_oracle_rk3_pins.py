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


# ---------------------------------------------------------------------------------------------
# Advection on the stretched grid: second-order convergence to the continuum -div(u u)
# ---------------------------------------------------------------------------------------------
ADV_L = (1.0, 0.7, 2.0)  # Lx, Ly, Lz


def _continuum_advection():
    """A smooth divergence-free channel field and its exact advection term -div(u u).

    With s(z) = 1 - cos(2 pi z / Lz) (s and s' vanish on both walls), a = 2 pi / Lx, b = 2 pi / Ly:
    w = s sin(ax) cos(by), u = U0(z) + s'/(2a) cos(ax) cos(by), v = V0(z) - s'/(2b) sin(ax) sin(by),
    so u_x + v_y = -s' sin(ax) cos(by) = -w_z, and u = v = w = 0 on the walls (no slip).  The exact
    derivatives come from sympy, independently of the oracle's stencils."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    lx, ly, lz = ADV_L
    a, b = 2 * sp.pi / lx, 2 * sp.pi / ly
    s = 1 - sp.cos(2 * sp.pi * z / lz)
    ds = sp.diff(s, z)
    u = sp.sin(sp.pi * z / lz) + ds / (2 * a) * sp.cos(a * x) * sp.cos(b * y)
    v = sp.Rational(3, 10) * sp.sin(2 * sp.pi * z / lz) - ds / (2 * b) * sp.sin(a * x) * sp.sin(b * y)
    w = s * sp.sin(a * x) * sp.cos(b * y)
    assert sp.simplify(sp.diff(u, x) + sp.diff(v, y) + sp.diff(w, z)) == 0
    adv = [-(sp.diff(c * u, x) + sp.diff(c * v, y) + sp.diff(c * w, z)) for c in (u, v, w)]
    f = lambda e: sp.lambdify((x, y, z), e, "numpy")
    return [f(e) for e in (u, v, w)], [f(e) for e in adv]


def advection_errors(n, fields=None):
    """Max error of the oracle's advection term (nu = 0) against the continuum one on an n^3 tanh grid
    (alpha 1.8), each component sampled at its own staggered location."""
    (fu, fv, fw), (au, av, aw) = fields or _continuum_advection()
    lx, ly, lz = ADV_L
    dzf = I.tanh_dzf(n, 1.8, lz)
    zf = np.concatenate([[0.0], np.cumsum(dzf)])
    zc = 0.5 * (zf[:-1] + zf[1:])
    xc, xf = (np.arange(n) + 0.5) * lx / n, (np.arange(n) + 1.0) * lx / n
    yc, yf = (np.arange(n) + 0.5) * ly / n, (np.arange(n) + 1.0) * ly / n

    def at(fn, zz, yy, xx):
        return np.broadcast_to(fn(xx[None, None, :], yy[None, :, None], zz[:, None, None]), (n, n, n)).copy()

    u, eu = at(fu, zc, yc, xf), at(au, zc, yc, xf)
    v, ev = at(fv, zc, yf, xc), at(av, zc, yf, xc)
    w, ew = at(fw, zf[1:], yc, xc), at(aw, zf[1:], yc, xc)
    w[-1] = 0.0
    ru, rv, rw = oracle.momentum_rhs(u, v, w, 0.0, ADV_L[:2], dzf)
    return np.array([np.abs(ru - eu).max(), np.abs(rv - ev).max(), np.abs(rw[:-1] - ew[:-1]).max()])


def advection_orders(fields=None):
    e = [advection_errors(n, fields) for n in (16, 32, 64)]
    return np.log2(e[1] / e[2]), e[2]


def test_advection_is_second_order_on_stretched_grid():
    """Every component of the advection term converges at second order on the tanh-stretched grid.

    A swapped z metric (cell width dzf where the centre distance dzc belongs, or the reverse) leaves a
    first-order error on a stretched grid, which this catches and the uniform-grid energy pin cannot."""
    orders, err64 = advection_orders()
    assert (orders > 1.75).all(), orders
    assert (err64 < 0.06).all(), err64


# ---------------------------------------------------------------------------------------------
# Stable time step: closed forms that isolate each row and each term of the inverse time scale
# ---------------------------------------------------------------------------------------------
DT_SHAPE = (10, 6, 8)  # (nz, ny, nx)


def dt_cases():
    """(name, (u, v, w), exact dt / cfl) on the stretched grid, cfl = 1 and negligible viscosity.

    A field alternating in sign along two directions cancels in every four-point average that spans
    one of them, so only the chosen row of Eq. dt's inverse time scale survives.  A w spike on one
    face k0 gives |w| / (distance between centres k0, k0+1) in the z row and |w| / (2 dzf) in the x and
    y rows of the two cells that share the face."""
    dzf = I.tanh_dzf(DT_SHAPE[0], 1.8, 2.0)
    dzc = 0.5 * (dzf[:-1] + dzf[1:])
    dx, dy = L[0] / DT_SHAPE[2], L[1] / DT_SHAPE[1]
    k, j, i = np.meshgrid(*(np.arange(n) for n in DT_SHAPE), indexing="ij")
    alt_jk, alt_ik = (-1.0) ** (j + k), (-1.0) ** (i + k)
    z = np.zeros(DT_SHAPE)
    k0 = 2  # lower half: dzf[k0] < dzf[k0 + 1]

    def spike(amp):
        w = np.zeros(DT_SHAPE)
        w[k0] = amp
        return w

    r3 = np.sqrt(3.0)
    return dzf, [
        ("v only", (z, 3 * alt_ik, z), r3 * dy / 3),
        ("w only", (z, z, spike(2.0)), r3 * dzc[k0] / 2),
        ("x row: u, v", (40 * alt_jk, np.full(DT_SHAPE, 3.0), z), r3 / (40 / dx + 3 / dy)),
        ("x row: u, w", (40 * alt_jk, z, spike(2.0)), r3 / (40 / dx + 1 / dzf[k0])),
        ("y row: v, w", (z, 40 * alt_ik, spike(2.0)), r3 / (40 / dy + 1 / dzf[k0])),
        ("y row: u, v", (np.full(DT_SHAPE, 2.0), 5 * alt_ik, z), r3 / (2 / dx + 5 / dy)),
        ("z row: u, w", (np.full(DT_SHAPE, 2.0), z, spike(2.0)), r3 / (2 / dx + 2 / dzc[k0])),
    ]


def dt_mismatches():
    dzf, cases = dt_cases()
    return {name: abs(oracle.stable_dt(*f, 1e-9, 1.0, L, dzf) - want) / want for name, f, want in cases}


def test_stable_dt_closed_forms_for_each_row():
    bad = {k: v for k, v in dt_mismatches().items() if v > 1e-14}
    assert not bad, bad


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
