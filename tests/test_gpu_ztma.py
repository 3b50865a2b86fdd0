"""The TMA-fed float z pass against the register-staged one and the oracle.

Both kernels run the same per-column arithmetic (zsolve_pair / zsolve_column on a bank-swizzled tile)
and differ only in how tiles reach shared memory (a tensor copy into a staging buffer on an mbarrier,
persistent CTAs, 16-slot tiles, against register-staged 16-byte loads) and in the swizzle, so mixed
solves through either must agree bit for bit; the TMA solve must also match the oracle (Eq.
poi_reduced) to the mixed path's bound.  CANS_Z_TMA=2 makes a plan fail rather than fall back, so
these cases are known to run the TMA kernel; the shapes cover 4, 8 and 16 rows per lane, column pairs
(x periodic) and single columns, FP64 low-|mu| columns inside TMA tiles, and more tiles than resident
CTAs (each CTA walks several tiles through its copy pipeline).
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


@pytest.mark.parametrize("n,bc", SHAPES)
def test_tma_z_pass_matches_staged_kernel_bitwise_and_oracle(cans, monkeypatch, n, bc):
    import torch

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
