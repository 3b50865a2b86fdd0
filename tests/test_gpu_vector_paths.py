"""Solves whose fields do not allow the passes' 16-byte vector accesses.

The fast kernels move 16-byte vectors (cp.async tile staging, float4 / double2 loads and stores) where
the row length and the addresses allow; otherwise each pass has an element-wise form.  These cases
force the element-wise forms and compare the solve with the oracle (Eq. poi_reduced): x lines whose
length is not a multiple of 4 (the y and z tiles of such a grid are not 16-byte rows), and f and p at
addresses that are 8- but not 16-byte aligned (legal for double arrays), on the FP64 path, which
transforms p in place, and on the mixed path, whose first x pass reads f and last x pass writes p.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD = 0, 1, 2


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def _check(cans, n, bc, length_xy, dzf, prec, f, fdev, pdev):
    import torch

    s = cans.PoissonSolver(n, bc, length_xy, dzf, prec=prec, sweeps=3)
    _, info, st = s.solve(fdev, out=pdev, info=True)
    torch.cuda.synchronize()
    s.close()
    assert st == 0, info
    ref = oracle.poisson_solve(f, bc, length_xy, dzf, nthreads=8)
    rel = float(np.linalg.norm(pdev.cpu().numpy() - ref) / np.linalg.norm(ref))
    assert rel <= (1e-12 if prec == 0 else 1e-10), rel


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,bc", [((6, 64, 16), (P, P, NN)), ((18, 48, 10), (NN, DD, DD)), ((54, 32, 12), (DD, P, NN))])
def test_x_lines_not_a_multiple_of_4(cans, prec, n, bc):
    import torch

    dzf = I.tanh_dzf(n[2], 1.5)
    case = I.PoissonCase("vec", n, bc, (1.0, 1.0), dzf, 4250, "uniform")
    f = I.rhs_host(case)
    ft = torch.from_numpy(f).cuda()
    _check(cans, n, bc, (1.0, 1.0), dzf, prec, f, ft, torch.empty_like(ft))


@pytest.mark.parametrize("prec", [0, 1])
def test_8_byte_aligned_f_and_p(cans, prec):
    import torch

    n, bc, length_xy = (256, 32, 40), (P, DD, NN), (1.0, 1.0)
    dzf = I.tanh_dzf(n[2], 1.8)
    case = I.PoissonCase("vec", n, bc, length_xy, dzf, 4244, "uniform")
    f = I.rhs_host(case)
    big = torch.empty(2 * f.size + 3, dtype=torch.float64, device="cuda")
    fm = big[1:1 + f.size].view(f.shape)
    pm = big[f.size + 3:].view(f.shape)
    fm.copy_(torch.from_numpy(f).cuda())
    assert fm.data_ptr() % 16 == 8 and pm.data_ptr() % 16 == 8
    _check(cans, n, bc, length_xy, dzf, prec, f, fm, pm)
