"""Robustness checks of the solver state handling: a workspace poisoned with NaN before each solve must
not change any result beyond the run-to-run order of the atomic reductions (no path reads workspace it
has not written), and the RK3 state is exactly the caller's (u, v, w, p): a checkpoint written to disk
and reloaded into a fresh plan continues the run (to the run-to-run order of the atomic sums)."""
import io

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


@pytest.mark.parametrize("n,bc,prec,shift,z_grid", [
    ((32, 24, 16), (0, 0, 1), 1, 0.0, 0),      # mixed, shared-memory engine, singular
    ((256, 256, 24), (0, 0, 1), 1, 0.0, 0),    # mixed, warp-per-line engine and streaming residual
    ((24, 18, 17), (3, 4, 2), 1, 0.0, 0),      # quarter-wave walls
    ((48, 32, 20), (1, 2, 2), 1, -50.0, 1),    # Helmholtz on the face grid
    ((32, 24, 16), (0, 0, 1), 0, 0.0, 0),      # FP64 (works in place, no workspace)
])
def test_nan_poisoned_workspace_changes_nothing(cans, n, bc, prec, shift, z_grid):
    import torch

    dzf = I.tanh_dzf(n[2], 1.5)
    f = torch.from_numpy(I.uniform(201, (n[2], n[1], n[0]), -1, 1)).cuda()
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=prec, sweeps=2, shift=shift, z_grid=z_grid)
    clean = torch.empty_like(f)
    s.workspace.zero_()
    s.solve(f, clean)
    poisoned = torch.empty_like(f)
    s.workspace[: s.workspace.numel() // 4 * 4].view(torch.float32).fill_(float("nan"))
    s.solve(f, poisoned)
    torch.cuda.synchronize()
    nu = n[2] - z_grid

    tol = 1e-13 if prec == 0 else 1e-10  # the order of the atomic reductions, within the method accuracy (max norm)

    def same(a, b):  # finite, and equal up to that order
        scale = float(b.abs().max())
        d = float((a - b).abs().max())
        assert bool(torch.isfinite(a).all()) and d <= tol * scale, (d, scale)
        return True

    assert same(poisoned[:nu], clean[:nu])
    # the adjoint's workspace as well
    g1 = s.solve_adjoint(f)
    s._adj_ws[: s._adj_ws.numel() // 4 * 4].view(torch.float32).fill_(float("nan"))
    g2 = s.solve_adjoint(f)
    torch.cuda.synchronize()
    assert same(g2[:nu], g1[:nu])
    s.close()


def test_rk3_checkpoint_restart_is_exact(cans):
    import torch

    shape, L = (16, 12, 16), (2.0, 1.0)
    dzf = I.tanh_dzf(16, 1.8, 2.0)
    zc = I.z_centres(dzf)
    u = 1.5 * (1 - (zc - 1) ** 2)[:, None, None] + 0.1 * I.uniform(211, shape, -1, 1)
    v = 0.1 * I.uniform(212, shape, -1, 1)
    w = 0.1 * I.uniform(213, shape, -1, 1)
    w[-1] = 0.0
    u, v, w = oracle.project(u, v, w, L, dzf)[:3]
    state = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (u, v, w, np.zeros(shape))]
    ch = cans.Channel((16, 12, 16), L, dzf, prec=cans.CANS_MIXED)
    straight = [t.clone() for t in state]
    for _ in range(4):
        ch.rk3_step(*straight, 0.002, cfl=0.9, ubulk=1.0)
    first = [t.clone() for t in state]
    for _ in range(2):
        ch.rk3_step(*first, 0.002, cfl=0.9, ubulk=1.0)
    ch.close()
    buf = io.BytesIO()
    torch.save([t.cpu() for t in first], buf)  # the checkpoint: the caller's four fields
    buf.seek(0)
    restored = [t.cuda() for t in torch.load(buf)]
    ch2 = cans.Channel((16, 12, 16), L, dzf, prec=cans.CANS_MIXED)  # a fresh plan from (n, bc, dzf)
    for _ in range(2):
        ch2.rk3_step(*restored, 0.002, cfl=0.9, ubulk=1.0)
    torch.cuda.synchronize()
    for a, b in zip(restored[:3], straight[:3]):  # equal up to the order of the atomic sums (bulk velocity)
        assert float((a - b).abs().max()) <= 1e-11 * float(b.abs().max())
    ch2.close()
