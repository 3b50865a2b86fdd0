"""GPU parity of the fractional-step path (RK3 step, projection, adjoint, autograd) against the oracle."""
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def channel_state(shape, L, dzf, seed, amp=0.1):
    """Laminar parabola + amp * U[-1,1] perturbation, w = 0 on the top wall face."""
    nz = shape[0]
    zc = I.z_centres(dzf)
    lz = float(dzf.sum())
    prof = 1.5 * (1 - (2 * zc / lz - 1) ** 2)
    u = prof[:, None, None] + amp * I.uniform(seed, shape, -1, 1, stream=11)
    v = amp * I.uniform(seed, shape, -1, 1, stream=12)
    w = amp * I.uniform(seed, shape, -1, 1, stream=13)
    w[-1] = 0.0
    return u, v, w


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-10)])
def test_rk3_step_matches_oracle(cans, prec, tol):
    import torch

    shape, L = (16, 24, 32), (4 * np.pi / 8, 2 * np.pi / 8)
    dzf = I.tanh_dzf(16, 1.8, 2.0)
    u, v, w = channel_state(shape, L, dzf, 5)
    u, v, w = oracle.project(u, v, w, L, dzf)[:3]
    p = np.zeros(shape)
    nu = 2.0 / 5600
    ch = cans.Channel((32, 24, 16), L, dzf, prec=prec)
    tu, tv, tw, tp = dev(u), dev(v), dev(w), dev(p)
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    ch.rk3_step(tu, tv, tw, tp, nu, cfl=0.9, ubulk=1.0, dt_out=dt_dev)
    ou, ov, ow, op, odt = oracle.rk3_step(u, v, w, p, nu, 0.9, 1.0, L, dzf)
    assert abs(float(dt_dev.item()) - odt) <= 1e-14 * odt
    for got, want in ((host(tu), ou), (host(tv), ov), (host(tw), ow)):
        assert rel(got, want) <= tol
    # pressure is defined up to a constant per substage gauge: compare the zero-mean parts
    gp, wp = host(tp), op
    wgt = dzf[:, None, None] * np.ones(shape)
    gp = gp - (gp * wgt).sum() / wgt.sum()
    wp = wp - (wp * wgt).sum() / wgt.sum()
    assert rel(gp, wp) <= 100 * tol
    ch.close()


def test_rk3_two_steps_and_fixed_dt(cans):
    shape, L = (8, 12, 16), (2.0, 1.0)
    dzf = I.tanh_dzf(8, 1.5, 2.0)
    u, v, w = oracle.project(*channel_state(shape, L, dzf, 7), L, dzf)[:3]
    p = np.zeros(shape)
    ch = cans.Channel((16, 12, 8), L, dzf)
    tu, tv, tw, tp = dev(u), dev(v), dev(w), dev(p)
    for _ in range(2):
        ch.rk3_step(tu, tv, tw, tp, 1e-2, dt=2e-3)
        u, v, w, p, _ = oracle.rk3_step(u, v, w, p, 1e-2, 0.9, 1.0, L, dzf, dt=2e-3)
    assert rel(host(tu), u) < 1e-11 and rel(host(tv), v) < 1e-11 and rel(host(tw), w) < 1e-11
    ch.close()


def test_projection_matches_oracle_and_is_divergence_free(cans):
    shape, L = (16, 12, 24), (1.5, 1.0)
    dzf = I.tanh_dzf(16, 1.8, 2.0)
    rng = np.random.default_rng(3)
    u, v, w = (rng.standard_normal(shape) for _ in range(3))
    w[-1] = 0
    ch = cans.Channel((24, 12, 16), L, dzf)
    tu, tv, tw = dev(u), dev(v), dev(w)
    ch.project_(tu, tv, tw)
    pu, pv, pw, _ = oracle.project(u, v, w, L, dzf)
    gu, gv, gw = host(tu), host(tv), host(tw)
    assert rel(gu, pu) < 1e-12 and rel(gv, pv) < 1e-12 and rel(gw, pw) < 1e-12
    assert np.abs(oracle.divergence(gu, gv, gw, L, dzf)).max() < 1e-10
    ch.close()


def test_adjoint_matches_dense_transpose(cans):
    """Assemble P column by column with the oracle on 6x4x4 and compare P^T with the GPU adjoint."""
    shape, L = (4, 4, 6), (1.0, 0.8)
    dzf = I.tanh_dzf(4, 1.4, 2.0)
    n = int(np.prod(shape))
    cols = []
    for comp in range(3):
        for c in range(n):
            e = [np.zeros(shape) for _ in range(3)]
            e[comp].flat[c] = 1.0
            e[2][-1] = 0.0
            cols.append(np.concatenate([a.ravel() for a in oracle.project(*e, L, dzf)[:3]]))
    Pm = np.array(cols).T  # (3n, 3n)
    rng = np.random.default_rng(9)
    g = rng.standard_normal(3 * n)
    g[2 * n:][-shape[1] * shape[2]:] = 0.0  # no component on the top wall face
    want = Pm.T @ g
    ch = cans.Channel((6, 4, 4), L, dzf)
    gu, gv, gw = (dev(g[k * n:(k + 1) * n].reshape(shape)) for k in range(3))
    ch.project_(gu, gv, gw, adjoint=True)
    got = np.concatenate([host(t).ravel() for t in (gu, gv, gw)])
    keep = np.ones(3 * n, bool)
    keep[2 * n:][-shape[1] * shape[2]:] = False  # wall face rows are identically zero
    assert np.abs(got[keep] - want[keep]).max() < 1e-11 * np.abs(want).max()
    ch.close()


def test_dot_product_adjoint_identity(cans):
    shape, L = (16, 16, 16), (1.0, 1.0)
    dzf = I.tanh_dzf(16, 1.8, 1.0)
    rng = np.random.default_rng(4)
    a = [rng.standard_normal(shape) for _ in range(3)]
    b = [rng.standard_normal(shape) for _ in range(3)]
    a[2][-1] = 0
    b[2][-1] = 0
    ch = cans.Channel((16, 16, 16), L, dzf)
    Pa = [dev(x) for x in a]
    ch.project_(*Pa)
    PTb = [dev(x) for x in b]
    ch.project_(*PTb, adjoint=True)
    lhs = sum(float((host(x) * y).sum()) for x, y in zip(Pa, b))
    rhs = sum(float((x * host(y)).sum()) for x, y in zip(a, PTb))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    ch.close()


def test_projection_gradient_matches_finite_differences(cans):
    """Loss = <g, P u*>: autograd (adjoint kernel) vs central differences on 16^3 along 8 directions."""
    import torch

    shape, L = (16, 16, 16), (1.0, 1.0)
    dzf = I.tanh_dzf(16, 1.8, 1.0)
    ch = cans.Channel((16, 16, 16), L, dzf)
    rng = np.random.default_rng(5)
    u0 = [dev(rng.standard_normal(shape)) for _ in range(3)]
    u0[2][-1] = 0
    g = [dev(rng.standard_normal(shape)) for _ in range(3)]

    def loss(u, v, w):
        pu, pv, pw = cans.projection(ch, u, v, w)
        return (pu * g[0]).sum() + (pv * g[1]).sum() + (pw * g[2]).sum()

    x = [t.clone().requires_grad_(True) for t in u0]
    lval = loss(*x)
    lval.backward()
    grads = [t.grad.detach() for t in x]
    for d in range(8):
        e = [dev(rng.standard_normal(shape)) for _ in range(3)]
        e[2][-1] = 0
        h = 1e-6 * float(torch.sqrt(sum((t * t).sum() for t in u0)))
        with torch.no_grad():
            lp = loss(*[a + h * b for a, b in zip(u0, e)])
            lm = loss(*[a - h * b for a, b in zip(u0, e)])
        fd = float((lp - lm) / (2 * h))
        ad = float(sum((gr * b).sum() for gr, b in zip(grads, e)))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (d, fd, ad)
    ch.close()


def test_rk3_step_in_cuda_graph_matches_eager(cans):
    import torch

    shape, L = (16, 16, 32), (2.0, 1.0)
    dzf = I.tanh_dzf(16, 1.8, 2.0)
    u, v, w = oracle.project(*channel_state(shape, L, dzf, 21), L, dzf)[:3]
    ch = cans.Channel((32, 16, 16), L, dzf, prec=1)
    eager = [dev(a) for a in (u, v, w, np.zeros(shape))]
    ch.rk3_step(*eager, 1e-3)
    graphed = [dev(a) for a in (u, v, w, np.zeros(shape))]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside the capture (sets kernel attributes)
        warm = [t.clone() for t in graphed]
        ch.rk3_step(*warm, 1e-3, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ch.rk3_step(*graphed, 1e-3)
    graph.replay()
    torch.cuda.synchronize()
    # identical kernels; only the order of the atomic bulk-velocity sum may differ between runs
    scale = max(float(b.abs().max()) for b in eager)
    for a, b in zip(graphed, eager):
        assert float((a - b).abs().max()) <= 1e-12 * scale
    ch.close()


@pytest.mark.slow
def test_config4_channel_step_matches_oracle(cans):
    """512x256x192 channel (Lx = 4 pi, Ly = 2 pi, Lz = 2, tanh 1.8, Re_b = 5600), one FP64 step."""
    import torch

    shape, L = (192, 256, 512), (4 * np.pi, 2 * np.pi)
    dzf = I.tanh_dzf(192, 1.8, 2.0)
    u, v, w = channel_state(shape, L, dzf, I.SEED_BASE + 4)
    p = np.zeros(shape)
    nu = 2.0 / 5600
    ch = cans.Channel((512, 256, 192), L, dzf)
    t = [dev(a) for a in (u, v, w, p)]
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    ch.rk3_step(*t, nu, cfl=0.9, ubulk=1.0, dt_out=dt_dev)
    ou, ov, ow, op, odt = oracle.rk3_step(u, v, w, p, nu, 0.9, 1.0, L, dzf)
    assert abs(float(dt_dev.item()) - odt) <= 1e-14 * odt
    for got, want in zip(t[:3], (ou, ov, ow)):
        assert rel(host(got), want) <= 1e-11
    ch.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-10)])
def test_rk3_step_implicit_matches_oracle(cans, prec, tol):
    """cans_rk3_step_implicit (Crank-Nicolson diffusion, Eq. up_id / up_id_2: three Helmholtz solves per
    substage, w on the interior z-faces) against the oracle's implicit step, a low-Reynolds channel
    with a fixed dt ten times the explicit viscous limit."""
    import torch

    shape, L = (16, 12, 24), (2.0, 1.0)
    dzf = I.tanh_dzf(16, 1.8, 2.0)
    u, v, w = channel_state(shape, L, dzf, 21)
    u, v, w = oracle.project(u, v, w, L, dzf)[:3]
    p = 0.05 * I.uniform(22, shape, -1, 1)
    nu = 0.05
    dl = min(L[0] / 24, L[1] / 12, float(dzf.min()))
    dt = 10 * 1.65 * dl * dl / nu
    ch = cans.Channel((24, 12, 16), L, dzf, prec=prec, implicit=True)
    tu, tv, tw, tp = dev(u), dev(v), dev(w), dev(p)
    for _ in range(2):
        ch.rk3_step_implicit(tu, tv, tw, tp, nu, dt, ubulk=1.0)
    ou, ov, ow, op = u, v, w, p
    for _ in range(2):
        ou, ov, ow, op, _ = oracle.rk3_step_implicit(ou, ov, ow, op, nu, 0.5, 1.0, L, dzf, dt=dt)
    for got, want in ((host(tu), ou), (host(tv), ov), (host(tw), ow)):
        assert rel(got, want) <= tol, rel(got, want)
    assert np.all(host(tw)[-1] == 0.0)
    gp, wp = host(tp), op
    wgt = dzf[:, None, None] * np.ones(shape)
    gp = gp - (gp * wgt).sum() / wgt.sum()
    wp = wp - (wp * wgt).sum() / wgt.sum()
    assert rel(gp, wp) <= 100 * tol, rel(gp, wp)
    d = oracle.divergence(host(tu), host(tv), host(tw), L, dzf)
    assert np.abs(d).max() <= 1e-9
    ch.close()


def test_rk3_step_implicit_argument_checks(cans):
    import torch

    shape, L = (8, 8, 8), (1.0, 1.0)
    dzf = I.tanh_dzf(8, 1.5, 2.0)
    ch = cans.Channel((8, 8, 8), L, dzf, implicit=True)
    t = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(4)]
    prm = cans.cans_rk3_params(0.1, 0.5, 1.0, 0.0, 1)  # dt = 0: the implicit step needs a fixed dt
    st = cans.cans_rk3_step_implicit(ch.plan, ch.uv_plan, ch.w_plan, *(x.data_ptr() for x in t), prm, 0, ch._im_ws, 0)
    assert st == cans.CANS_ERR_ARG
    prm = cans.cans_rk3_params(0.1, 0.5, 1.0, 1e-3, 1)
    st = cans.cans_rk3_step_implicit(ch.plan, ch.w_plan, ch.uv_plan, *(x.data_ptr() for x in t), prm, 0, ch._im_ws, 0)
    assert st == cans.CANS_ERR_ARG  # plans swapped
    ch.close()
