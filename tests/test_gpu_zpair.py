"""The float z pass on pair-granular tiles against the staged kernel and the oracle.

For a periodic x direction the Re / Im slots of one wavenumber share their z system (Eq. poi_reduced
with equal mu); with walls in x every column has its own.  The pair-granular kernel keeps the columns
2p and 2p + 1 side by side, fetches its
tiles with 8-byte cp.async copies and solves each pair with both right-hand sides of a row in one
8-byte word; the arithmetic per column is the staged kernel's, so mixed solves through either must
agree bit for bit (CANS_Z_P2=0 selects the staged kernel), and both must match the oracle.  The shapes
take 4, 8 and 16 rows per lane (Nz = 128, 256, 512), slot 0 and 1 of x (solved as single columns), the
low-|mu| columns left to the double kernel, Neumann, Dirichlet and mixed y walls, and a Helmholtz shift.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD, ND = 0, 1, 2, 3

CASES = [
    # n, bc, length_xy, shift
    ((256, 48, 512), (P, P, NN), (256 / 1024, 48 / 1024), 0.0),   # 16 rows per lane, singular
    ((128, 64, 256), (P, DD, NN), (1.0, 1.0), 0.0),               # 8 rows per lane
    ((64, 48, 128), (P, NN, DD), (1.0, 0.5), 0.0),                # 4 rows per lane, Dirichlet z
    ((96, 24, 512), (P, ND, NN), (1.0, 1.0), -30.0),              # mixed y walls, shift, three tiles in x
    # walled x: every column solved on its own from the pair-granular tile
    ((128, 48, 512), (NN, P, NN), (1.0, 1.0), 0.0),               # singular
    ((64, 32, 256), (DD, DD, NN), (1.0, 1.0), 0.0),
    ((96, 24, 128), (ND, NN, DD), (1.0, 0.5), -10.0),             # quarter-wave x, shift
    ((32, 48, 512), (4, P, NN), (32 / 1024, 48 / 1024), 0.0),     # quarter-wave x (Dirichlet first), one tile
]


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


@pytest.mark.parametrize("n,bc,length_xy,shift", CASES)
def test_pair_tiles_match_staged_kernel_bitwise_and_oracle(cans, monkeypatch, n, bc, length_xy, shift):
    import torch

    dzf = I.tanh_dzf(n[2], 1.7)
    case = I.PoissonCase("zp", n, bc, length_xy, dzf, 4270, "uniform")
    f = I.rhs_host(case)
    ft = torch.from_numpy(f).cuda()
    got = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("CANS_Z_P2", flag)
        s = cans.PoissonSolver(n, bc, length_xy, dzf, prec=1, sweeps=2, shift=shift)
        p, info, st = s.solve(ft, info=True)
        torch.cuda.synchronize()
        got[flag] = (p.cpu().numpy(), info, st)
        s.close()
    p2, info, st = got["1"]
    assert st == 0, info
    assert np.array_equal(p2, got["0"][0])
    ref = oracle.helmholtz_solve(f, bc, length_xy, dzf, shift=shift, nthreads=8)
    rel = float(np.linalg.norm(p2 - ref) / np.linalg.norm(ref))
    assert rel <= 1e-10, rel


def test_pair_tiles_first_solve_matches_staged_kernel(cans, monkeypatch):
    """No refinement sweep: the first float solve itself (the z pass's own rounding shows) is equal."""
    import torch

    n, bc = (128, 32, 512), (P, P, NN)
    dzf = I.tanh_dzf(512, 1.8)
    case = I.PoissonCase("zp", n, bc, (1.0, 1.0), dzf, 4271, "uniform")
    ft = torch.from_numpy(I.rhs_host(case)).cuda()
    got = []
    for flag in ("1", "0"):
        monkeypatch.setenv("CANS_Z_P2", flag)
        s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=0)
        got.append(s.solve(ft).cpu().numpy())
        s.close()
    assert np.array_equal(got[0], got[1])
