"""cans_poisson_solve_divergence: Eq. poi_ns with its right-hand side f = D(u*) / (gamma dt) formed
inside the solve's first x pass.

Its f (written as a by-product) must match the oracle's divergence of the same face fields, and its
p must equal, bit for bit, cans_poisson_solve applied to that f (the divergence takes the roundings
of the stand-alone kernel), on the warp-per-line x kernels (periodic lines of 256 / 512 / 1024 points)
and on the CTA-wide ones (other lengths, and every FP64 plan).
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN = 0, 1


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def _fields(n, seed=3):
    rng = np.random.default_rng(seed)
    shape = (n[2], n[1], n[0])
    u, v, w = (rng.standard_normal(shape) for _ in range(3))
    w[-1] = 0.0  # the top wall face
    return u, v, w


@pytest.mark.parametrize("prec,sweeps", [(0, 0), (1, 1), (1, 2)])
@pytest.mark.parametrize("n", [(256, 64, 24), (48, 32, 20), (512, 16, 8)])
def test_fused_divergence_solve_matches_two_step_solve(cans, prec, sweeps, n):
    import torch

    L = (4 * np.pi, 2 * np.pi)
    dzf = I.tanh_dzf(n[2], 1.8, 2.0)
    u, v, w = _fields(n)
    ut, vt, wt = (torch.from_numpy(a).cuda() for a in (u, v, w))
    gamma, dt = 8.0 / 15.0, 3.7e-3
    dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
    s = cans.PoissonSolver(n, (P, P, NN), L, dzf, prec=prec, sweeps=sweeps)
    f = torch.empty_like(ut)
    p = torch.empty_like(ut)
    stream = int(torch.cuda.current_stream().cuda_stream)
    st = cans.cans_poisson_solve_divergence(s.plan, ut.data_ptr(), vt.data_ptr(), wt.data_ptr(), 1.0, dtt.data_ptr(),
                                            gamma, f.data_ptr(), p.data_ptr(), s._ws_ptr, stream)
    assert st == 0
    q = s.solve(f.clone())
    torch.cuda.synchronize()
    fh = f.cpu().numpy()
    want_f = oracle.divergence(u, v, w, L, dzf) / (gamma * dt)
    assert np.abs(fh - want_f).max() <= 1e-13 * np.abs(want_f).max()
    assert torch.equal(p, q)
    if prec == 0:  # FP64: f is optional and the result does not depend on it being written
        p2 = torch.empty_like(ut)
        st = cans.cans_poisson_solve_divergence(s.plan, ut.data_ptr(), vt.data_ptr(), wt.data_ptr(), 1.0,
                                                dtt.data_ptr(), gamma, 0, p2.data_ptr(), s._ws_ptr, stream)
        torch.cuda.synchronize()
        assert st == 0 and torch.equal(p2, p)
        ref = oracle.poisson_solve(want_f, (P, P, NN), L, dzf)
        assert np.linalg.norm(p.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    s.close()


def test_fused_divergence_solve_argument_checks(cans):
    import torch

    n = (32, 16, 8)
    dzf = I.uniform_dzf(8, 2.0)
    t = torch.zeros((8, 16, 32), dtype=torch.float64, device="cuda")
    f, p = torch.zeros_like(t), torch.zeros_like(t)
    stream = int(torch.cuda.current_stream().cuda_stream)
    mixed = cans.PoissonSolver(n, (P, P, NN), (1.0, 1.0), dzf, prec=1, sweeps=1)
    # the mixed refinement re-reads f: it must be given
    assert cans.cans_poisson_solve_divergence(mixed.plan, t.data_ptr(), t.data_ptr(), t.data_ptr(), 1.0, 0, 1.0, 0,
                                              p.data_ptr(), mixed._ws_ptr, stream) == -1
    # f may not alias a velocity or p
    assert cans.cans_poisson_solve_divergence(mixed.plan, t.data_ptr(), t.data_ptr(), t.data_ptr(), 1.0, 0, 1.0,
                                              t.data_ptr(), p.data_ptr(), mixed._ws_ptr, stream) == -1
    mixed.close()
    box = cans.PoissonSolver(n, (NN, P, NN), (1.0, 1.0), dzf, prec=0)
    assert cans.cans_poisson_solve_divergence(box.plan, t.data_ptr(), t.data_ptr(), t.data_ptr(), 1.0, 0, 1.0,
                                              f.data_ptr(), p.data_ptr(), 0, stream) == -2
    box.close()
