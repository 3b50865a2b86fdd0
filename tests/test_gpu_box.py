"""GPU parity of cans_box_rk3_step (the fractional step in a box with periodic or no-slip walled
directions and a moving lid) against the oracle's box step: lid-driven cavity, square duct, the
periodic Taylor-Green box, and the channel, where it must also agree with cans_rk3_step."""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu


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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def state(shape, walls, L, dzf, seed, amp=0.2, base=0.0):
    u = base + amp * I.uniform(seed, shape, -1, 1)
    v = amp * I.uniform(seed + 1, shape, -1, 1)
    w = amp * I.uniform(seed + 2, shape, -1, 1)
    for a, d in ((u, 2), (v, 1), (w, 0)):
        if walls[2 - d]:
            idx = [slice(None)] * 3
            idx[d] = -1
            a[tuple(idx)] = 0.0
    return oracle.box_project(u, v, w, walls, L, dzf)


CASES = {
    "cavity_lid": ((1, 1, 1), 1.0, False, 0.0),
    "duct_forced": ((0, 1, 1), 0.0, True, 1.0),
    "periodic": ((0, 0, 0), 0.0, False, 0.0),
    "channel": ((0, 0, 1), 0.0, True, 1.0),
    "walls_x_z": ((1, 0, 1), 0.0, False, 0.0),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-10)])
def test_box_step_matches_oracle(cans, name, prec, tol):
    walls, lid, forcing, ubulk = CASES[name]
    shape, L = (12, 12, 16), (1.5, 1.0)
    dzf = I.tanh_dzf(12, 1.6) if walls[2] else np.full(12, 1.0 / 12)
    u, v, w = state(shape, walls, L, dzf, 31, base=(1.0 if forcing else 0.0))
    p = 0.05 * I.uniform(34, shape, -1, 1)
    nu = 0.01
    box = cans.Box((16, 12, 12), L, dzf, walls, prec=prec)
    tu, tv, tw, tp = dev(u), dev(v), dev(w), dev(p)
    import torch

    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        box.rk3_step(tu, tv, tw, tp, nu, cfl=0.5, ubulk=ubulk, forcing=forcing, lid=lid, dt_out=dt_dev)
    ou, ov, ow, op = u, v, w, p
    for _ in range(2):
        ou, ov, ow, op, odt = oracle.box_rk3_step(ou, ov, ow, op, walls, nu, L, dzf, cfl=0.5, ubulk=ubulk,
                                                  forcing=forcing, lid=lid)
    assert abs(float(dt_dev.item()) - odt) <= 1e-12 * odt
    for got, want in ((host(tu), ou), (host(tv), ov), (host(tw), ow)):
        assert np.abs(got - want).max() <= tol * max(1.0, np.abs(want).max())
    gp, wp = host(tp), op
    wgt = dzf[:, None, None] * np.ones(shape)
    gp = gp - (gp * wgt).sum() / wgt.sum()
    wp = wp - (wp * wgt).sum() / wgt.sum()
    assert rel(gp, wp) <= 100 * tol
    assert np.abs(oracle.box_divergence(host(tu), host(tv), host(tw), walls, L, dzf)).max() <= 1e-9
    box.close()


def test_box_channel_equals_the_channel_step(cans):
    """With walls in z only the box step and the tuned channel step are the same method."""
    import torch

    shape, L = (16, 12, 16), (2.0, 1.0)
    dzf = I.tanh_dzf(16, 1.8, 2.0)
    u, v, w = state(shape, (0, 0, 1), L, dzf, 41, base=1.0)
    p = np.zeros(shape)
    a = [dev(x) for x in (u, v, w, p)]
    b = [dev(x) for x in (u, v, w, p)]
    box = cans.Box((16, 12, 16), L, dzf, (0, 0, 1))
    ch = cans.Channel((16, 12, 16), L, dzf)
    box.rk3_step(*a, 0.002, cfl=0.9, ubulk=1.0, forcing=True)
    ch.rk3_step(*b, 0.002, cfl=0.9, ubulk=1.0)
    for x, y in zip(a[:3], b[:3]):
        assert float((x - y).abs().max()) <= 1e-12 * float(y.abs().max())
    box.close()
    ch.close()


def test_taylor_green_vortex_decay(cans):
    """The periodic box: a Taylor-Green vortex of small amplitude decays like exp(-2 nu k_h^2 t) with the
    discrete wavenumber k_h^2 = (4/h^2) sin^2(h/2), over 40 steps (RK3 error O(dt^3) per step)."""
    import torch

    n = 32
    h = 2 * np.pi / n
    nz = 4
    xf, xc = (np.arange(n) + 1) * h, (np.arange(n) + 0.5) * h
    U = 1e-4
    u = U * np.sin(xf)[None, None, :] * np.cos(xc)[None, :, None] * np.ones((nz, 1, 1))
    v = -U * np.cos(xc)[None, None, :] * np.sin(xf)[None, :, None] * np.ones((nz, 1, 1))
    w = np.zeros_like(u)
    p = np.zeros_like(u)
    nu, dt, steps = 0.05, 0.02, 40
    box = cans.Box((n, n, nz), (2 * np.pi, 2 * np.pi), np.full(nz, 1.0 / nz), (0, 0, 0))
    t = [dev(x) for x in (u, v, w, p)]
    for _ in range(steps):
        box.rk3_step(*t, nu, dt=dt)
    kh2 = 4 / h ** 2 * np.sin(h / 2) ** 2
    decay = np.exp(-2 * nu * kh2 * dt * steps)
    got = host(t[0])
    assert np.abs(got - decay * u).max() <= 1e-6 * U
    box.close()
