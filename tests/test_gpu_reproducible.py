"""Run-to-run reproducibility of results that depend on grid-wide sums.

Two sums over the whole grid feed back into results: the dzf-weighted gauge sum of the mixed path's
first iterate, which fixes the mean of a singular solution (the all-periodic / Neumann column of
Eq. poi_reduced), and the bulk velocity of the constant-flow-rate forcing of the RK3 step (Eq. up).
Both are reduced with one slot per block and a fixed summation order, so repeating a solve or a step
from the same input reproduces every bit, however the blocks were scheduled.
"""
import numpy as np
import pytest

from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN = 0, 1


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


@pytest.mark.parametrize("n,length_xy", [((256, 16, 150), (256 / 1024, 16 / 1024)), ((96, 48, 40), (1.0, 1.0))])
def test_singular_mixed_solve_repeats_bit_for_bit(cans, n, length_xy):
    """The warp-engine path (Nx = 256) and the CTA-wide path (Nx = 96), x and y periodic, z Neumann."""
    import torch

    dzf = I.tanh_dzf(n[2], 1.6)
    case = I.PoissonCase("rep", n, (P, P, NN), length_xy, dzf, 4260, "uniform")
    ft = torch.from_numpy(I.rhs_host(case)).cuda()
    s = cans.PoissonSolver(n, (P, P, NN), length_xy, dzf, prec=1, sweeps=2)
    first = s.solve(ft).cpu().numpy()
    for _ in range(4):
        assert np.array_equal(s.solve(ft).cpu().numpy(), first)
    s.close()


def test_rk3_step_with_forcing_repeats_bit_for_bit(cans):
    """Two RK3 steps of a channel with the constant-flow-rate forcing, twice from the same state."""
    import torch

    shape, L = (16, 24, 32), (4 * np.pi / 8, 2 * np.pi / 8)
    dzf = I.tanh_dzf(16, 1.8, 2.0)
    zc = I.z_centres(dzf)
    prof = 1.5 * (1 - (2 * zc / float(dzf.sum()) - 1) ** 2)
    u0 = prof[:, None, None] + 0.1 * I.uniform(4261, shape, -1, 1, stream=11)
    v0 = 0.1 * I.uniform(4261, shape, -1, 1, stream=12)
    w0 = 0.1 * I.uniform(4261, shape, -1, 1, stream=13)
    w0[-1] = 0.0
    ch = cans.Channel((32, 24, 16), L, dzf, prec=1)
    runs = []
    for _ in range(2):
        u, v, w = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (u0, v0, w0))
        p = torch.zeros_like(u)
        for _ in range(2):
            ch.rk3_step(u, v, w, p, 1.0 / 5600, forcing=True, ubulk=1.0)
        torch.cuda.synchronize()
        runs.append([t.cpu().numpy() for t in (u, v, w, p)])
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    ch.close()
