"""The refinement residual's streaming stencil with four, two and one x-points per thread.

The mixed path's sweep residual r = f - L_h(Phi + Plo) (Eq. poi, with the Helmholtz shift of
Eq. up_id_2 when the plan has one) runs as a z-marching stencil where the x lines take the warp
engine.  The three thread shapes share the per-point double-float arithmetic, so solves through any of
them must agree bit for bit, and with the oracle to the mixed path's bound.  CANS_RES_PTS picks the
shape at plan creation; the cases cover the iso (dx = dy) and general x-y forms, the Plo term of later
sweeps, Neumann, Dirichlet, periodic and mixed walls in every direction, a Helmholtz shift, a ragged
last z chunk (Nz = 150 against chunks of 64 planes), and an f whose address is only 8-byte aligned
(every shape then falls back to one point per thread).
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD, ND, DN = 0, 1, 2, 3, 4

CASES = [
    # n, bc, length_xy, shift, sweeps
    ((256, 64, 40), (P, P, NN), (256 / 1024, 64 / 1024), 0.0, 2),     # iso, the bench's form, Plo sweep
    ((512, 48, 24), (NN, DD, DD), (1.0, 1.0), -50.0, 2),              # general x-y form, shift, walls
    ((1024, 24, 16), (DD, NN, P), (1.0, 0.5), 0.0, 3),                # periodic z wrap, three sweeps
    ((256, 36, 30), (ND, DN, ND), (1.0, 1.0), 0.0, 2),                # one Neumann and one Dirichlet wall
    ((256, 16, 150), (P, P, NN), (256 / 1024, 16 / 1024), 0.0, 2),    # ragged last z chunk
]


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def _solve(cans, monkeypatch, pts, n, bc, length_xy, dzf, shift, sweeps, ft):
    import torch

    monkeypatch.setenv("CANS_RES_PTS", pts)
    s = cans.PoissonSolver(n, bc, length_xy, dzf, prec=1, sweeps=sweeps, shift=shift)
    p, info, st = s.solve(ft, info=True)
    torch.cuda.synchronize()
    s.close()
    return p.cpu().numpy(), info, st


@pytest.mark.parametrize("n,bc,length_xy,shift,sweeps", CASES)
def test_residual_thread_shapes_agree_bitwise_and_with_oracle(cans, monkeypatch, n, bc, length_xy, shift, sweeps):
    import torch

    dzf = I.uniform_dzf(n[2]) if bc[2] == P else I.tanh_dzf(n[2], 1.6)  # a periodic z is uniform
    case = I.PoissonCase("res", n, bc, length_xy, dzf, 4242, "uniform")
    f = I.rhs_host(case)
    ft = torch.from_numpy(f).cuda()
    got = {pts: _solve(cans, monkeypatch, pts, n, bc, length_xy, dzf, shift, sweeps, ft) for pts in ("4", "2", "1")}
    p4, info, st = got["4"]
    assert st == 0, info
    assert np.array_equal(p4, got["2"][0])
    assert np.array_equal(p4, got["1"][0])
    ref = oracle.helmholtz_solve(f, bc, length_xy, dzf, shift=shift, nthreads=8)
    rel = float(np.linalg.norm(p4 - ref) / np.linalg.norm(ref))
    assert rel <= 1e-10, rel


def test_misaligned_f_falls_back_to_one_point_per_thread(cans, monkeypatch):
    """f at an address that is 8- but not 16-byte aligned: whatever CANS_RES_PTS asks, the stencil
    takes one point per thread (the first x pass also leaves the warp engine for the CTA-wide one), so
    the solves with 4 and with 1 agree bit for bit, reach the aligned solve's residuals, and match the
    oracle."""
    import torch

    n, bc, length_xy = (256, 64, 40), (P, P, NN), (256 / 1024, 64 / 1024)
    dzf = I.tanh_dzf(n[2], 1.6)
    case = I.PoissonCase("res", n, bc, length_xy, dzf, 4242, "uniform")
    f = I.rhs_host(case)
    big = torch.empty(f.size + 1, dtype=torch.float64, device="cuda")
    fm = big[1:].view(f.shape)
    fm.copy_(torch.from_numpy(f).cuda())
    assert fm.data_ptr() % 16 == 8
    pa = _solve(cans, monkeypatch, "4", n, bc, length_xy, dzf, 0.0, 2, torch.from_numpy(f).cuda())
    p4 = _solve(cans, monkeypatch, "4", n, bc, length_xy, dzf, 0.0, 2, fm)
    p1 = _solve(cans, monkeypatch, "1", n, bc, length_xy, dzf, 0.0, 2, fm)
    msg = (pa[1], pa[2], p4[1], p4[2])
    assert pa[2] == 0 and p4[2] == 0 and p1[2] == 0, msg
    assert np.array_equal(p4[0], p1[0])
    assert float(np.linalg.norm(p4[0] - pa[0]) / np.linalg.norm(pa[0])) <= 1e-11, msg
    ref = oracle.poisson_solve(f, bc, length_xy, dzf, nthreads=8)
    rel = float(np.linalg.norm(p4[0] - ref) / np.linalg.norm(ref))
    assert rel <= 1e-10, (rel, msg)


CTA_CASES = [
    # x lengths of the CTA-wide engine: the sweep residual as the streaming stencil + the float x pass
    ((96, 48, 40), (P, P, NN), (1.0, 1.0), 0.0, 2),
    ((48, 64, 32), (NN, DD, DD), (1.0, 0.5), -20.0, 2),
    ((192, 24, 16), (DD, NN, P), (1.0, 1.0), 0.0, 3),
    ((64, 32, 30), (ND, P, NN), (1.0, 1.0), 0.0, 2),
]


@pytest.mark.parametrize("n,bc,length_xy,shift,sweeps", CTA_CASES)
def test_split_residual_on_cta_engine_lines(cans, monkeypatch, n, bc, length_xy, shift, sweeps):
    """CTA-engine x lines: the split residual (stencil + in-place float x pass; CANS_RES_SPLIT=2 takes it
    at every size, by default only large fields do) against the oracle, and against the residual fused
    into the x pass (CANS_RES_SPLIT=0; the two round differently)."""
    import torch

    dzf = I.uniform_dzf(n[2]) if bc[2] == P else I.tanh_dzf(n[2], 1.6)
    case = I.PoissonCase("res", n, bc, length_xy, dzf, 4245, "uniform")
    f = I.rhs_host(case)
    ft = torch.from_numpy(f).cuda()
    got = {}
    for flag in ("2", "0"):  # split at every size / fused
        monkeypatch.setenv("CANS_RES_SPLIT", flag)
        got[flag] = _solve(cans, monkeypatch, "4", n, bc, length_xy, dzf, shift, sweeps, ft)
    ps, info, st = got["2"]
    assert st == 0, info
    ref = oracle.helmholtz_solve(f, bc, length_xy, dzf, shift=shift, nthreads=8)
    rel = float(np.linalg.norm(ps - ref) / np.linalg.norm(ref))
    assert rel <= 1e-10, rel
    pf = got["0"][0]
    assert float(np.linalg.norm(ps - pf) / np.linalg.norm(pf)) <= 1e-10
