"""The low-|mu| (and singular) z columns of short columns solved in FP64 inside the float z kernel.

For columns of at most 4 rows per lane on the staged float kernel, the kernel can solve its tile's
marked columns in FP64 itself (Eq. poi_reduced; the 1 % smallest-|mu| modes and the singular mode)
instead of leaving them to a second kernel -- by default on fields of up to 2^16 points, with
CANS_Z_FUSE64=2 at every size (the bit-for-bit comparison below).  The arithmetic per column is the double kernel's on the same tile
values, so mixed solves with and without the fusion (CANS_Z_FUSE64=0) agree bit for bit, and both match
the oracle; the singular column's compatibility sum still reaches the status word.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD = 0, 1, 2
INCOMPATIBLE = -5

CASES = [
    ((32, 32, 32), (P, P, NN), "uniform"),    # 1 row per lane, singular (gauge and compatibility sum)
    ((48, 24, 60), (NN, DD, NN), "tanh"),     # 2 rows per lane
    ((96, 64, 100), (P, NN, DD), "tanh"),     # 4 rows per lane, identity rows, column pairs
    ((24, 48, 128), (DD, P, NN), "tanh"),     # 4 rows per lane, x lines too short for the pair tile
]


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


@pytest.mark.parametrize("n,bc,z", CASES)
def test_fused_f64_columns_match_separate_kernel_bitwise_and_oracle(cans, monkeypatch, n, bc, z):
    import torch

    dzf = I.uniform_dzf(n[2]) if z == "uniform" else I.tanh_dzf(n[2], 1.5)
    case = I.PoissonCase("zf", n, bc, (1.0, 1.0), dzf, 4310, "uniform")
    f = I.rhs_host(case)
    ft = torch.from_numpy(f).cuda()
    got = {}
    for flag in ("2", "0"):  # fused at every size / the separate kernel
        monkeypatch.setenv("CANS_Z_FUSE64", flag)
        s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=2)
        p, info, st = s.solve(ft, info=True)
        torch.cuda.synchronize()
        got[flag] = (p.cpu().numpy(), info, st)
        s.close()
    pf, info, st = got["2"]
    assert st == 0, info
    assert np.array_equal(pf, got["0"][0])
    ref = oracle.poisson_solve(f, bc, (1.0, 1.0), dzf, nthreads=8)
    rel = float(np.linalg.norm(pf - ref) / np.linalg.norm(ref))
    assert rel <= 1e-11, rel


def test_fused_singular_column_reports_incompatible_rhs(cans, monkeypatch):
    """The singular column solved inside the float kernel still yields the compatibility check."""
    import torch

    monkeypatch.setenv("CANS_Z_FUSE64", "1")  # 32^3: fused by default
    n, bc = (32, 32, 32), (P, P, NN)
    dzf = I.uniform_dzf(32)
    case = I.PoissonCase("zf", n, bc, (1.0, 1.0), dzf, 4311, "uniform")
    f = I.rhs_host(case) + 0.5  # a nonzero mean: incompatible
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=1)
    s.solve(torch.from_numpy(f).cuda())
    assert s.status() == INCOMPATIBLE
    s.close()
