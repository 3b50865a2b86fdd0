"""The TMA-using float z kernels against the register-staged one and the oracle.

All variants run the same per-column arithmetic (zsolve_pair / zsolve_column on a bank-swizzled tile)
and differ only in how tiles reach shared memory: the register-staged kernel with a tensor prefetch
of a later tile into L2 (shape 4), or a tensor copy into a staging buffer on an mbarrier with
persistent CTAs -- one 512-thread CTA per SM on 32-slot tiles (shape 1), two or three 256-thread CTAs
on 16-slot tiles (2, 3).  Mixed solves through any of them must agree bit for bit with the
register-staged kernel, and match the oracle (Eq. poi_reduced) to the mixed path's bound.
CANS_Z_TMA=2 makes a plan fail rather than fall back, so these cases are known to run the chosen
kernel; the shapes cover 4, 8 and 16 rows per lane, column pairs (x periodic) and single columns,
FP64 low-|mu| columns inside the tiles (whose stores skip them), and more tiles than resident CTAs.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD = 0, 1, 2

SHAPES = [
    ((256, 64, 128), (P, P, NN)),     # 4 rows per lane, pairs, 1024 tiles
    ((128, 48, 256), (NN, P, NN)),    # 8 rows per lane, single columns
    ((1024, 16, 512), (P, DD, NN)),   # 16 rows per lane, pairs, 1024 tiles
    ((96, 48, 512), (DD, NN, DD)),    # 16 rows per lane, single columns, Dirichlet z
    ((64, 32, 512), (P, P, NN)),      # the singular mode inside a TMA tile (its column in FP64)
]


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


# 4: the register-staged kernel with the TMA prefetch of a later tile into L2; 1: tiles copied by TMA,
# one 512-thread CTA per SM (32-slot tiles); 2, 3: two or three 256-thread CTAs per SM (16-slot tiles)
@pytest.mark.parametrize("shape", ["4", "1", "2", "3"])
@pytest.mark.parametrize("n,bc", SHAPES)
def test_tma_z_pass_matches_staged_kernel_bitwise_and_oracle(cans, monkeypatch, n, bc, shape):
    import torch

    monkeypatch.setenv("CANS_Z_TMA_CTAS", shape)
    case = I.case_modes(n=n)
    case.bc = bc
    case.length_xy = (n[0] / 1024, n[1] / 1024)  # the bench's spacing
    case.dzf = I.tanh_dzf(n[2], 1.8)
    f = I.rhs_host(case)
    ft = torch.from_numpy(f).cuda()
    got = {}
    for flag in ("2", "0"):
        monkeypatch.setenv("CANS_Z_TMA", flag)
        s = cans.PoissonSolver(n, bc, case.length_xy, case.dzf, prec=1, sweeps=2)
        p, info, st = s.solve(ft, info=True)
        torch.cuda.synchronize()
        got[flag] = (p.cpu().numpy(), info, st)
        s.close()
    p_tma, info, st = got["2"]
    assert st == 0, info
    assert np.array_equal(p_tma, got["0"][0])
    # the solve met its 1e-12 residual (st == 0); the error that residual leaves depends on the
    # shape's conditioning: at most ~1e-11 here
    ref = oracle.poisson_solve(f, bc, case.length_xy, case.dzf, nthreads=8)
    rel = float(np.linalg.norm(p_tma - ref) / np.linalg.norm(ref))
    assert rel <= 1e-10, rel


def test_tma_required_on_a_shape_it_cannot_take_fails(cans, monkeypatch):
    """Nz = 200 (not full columns) with the TMA kernel required: the solve reports an error."""
    import torch

    monkeypatch.setenv("CANS_Z_TMA", "2")
    n = (64, 16, 200)
    dzf = I.tanh_dzf(200, 1.8)
    s = cans.PoissonSolver(n, (P, P, NN), (1.0, 1.0), dzf, prec=1, sweeps=1)
    f = torch.zeros((200, 16, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(cans.CansError):
        s.solve(f)
    s.close()
