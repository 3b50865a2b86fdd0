"""Full-size checks in the configuration bench.py times.

At 1024x1024x512 (mixed precision, one refinement sweep, autotuned plan, exactly as the bench) and
at the 1024x512x256 channel (FP64) the oracle's dense-basis solve is out of reach, so the checks are
properties that hold at any size: the oracle's own 7-point operator applied to the GPU solution on
the host (relative residual against f), and the agreement of the mixed and FP64 GPU solutions
(both in the zero dzf-weighted-mean gauge).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def test_bench_workload_mixed_full_size(cans):
    import torch

    case = I.case_modes()  # 1024 x 1024 x 512, x, y periodic, z Neumann on tanh faces
    f = I.rhs_device(case, "cuda")
    p = torch.empty_like(f)
    s = cans.PoissonSolver(case.n, case.bc, case.length_xy, case.dzf, prec=cans.CANS_MIXED, sweeps=1, autotune=True)
    _, info, st = s.solve(f, p, info=True)
    s.close()
    assert st == 0 and info[-1] <= 1e-12, info
    p64 = torch.empty_like(f)
    s64 = cans.PoissonSolver(case.n, case.bc, case.length_xy, case.dzf, prec=cans.CANS_FP64)
    s64.solve(f, p64)
    s64.close()
    torch.cuda.synchronize()
    diff = float(torch.linalg.vector_norm(p - p64) / torch.linalg.vector_norm(p64))
    assert diff <= 1e-11, diff
    del p64
    torch.cuda.empty_cache()
    fh, ph = f.cpu().numpy(), p.cpu().numpy()
    del f, p
    res = oracle.relative_residual(ph, fh, case.bc, case.length_xy, case.dzf, nthreads=os.cpu_count() or 1)
    assert res <= 1e-12, (res, info)


def test_channel_fp64_full_size(cans):
    import torch

    case = I.case_channel()  # 1024 x 512 x 256, x periodic, y Dirichlet, z Neumann on tanh faces
    f = I.rhs_device(case, "cuda")
    p = torch.empty_like(f)
    s = cans.PoissonSolver(case.n, case.bc, case.length_xy, case.dzf, prec=cans.CANS_FP64, autotune=True)
    _, info, st = s.solve(f, p, info=True)
    s.close()
    assert st == 0 and info[0] <= 1e-13, info
    fh, ph = f.cpu().numpy(), p.cpu().numpy()
    res = oracle.relative_residual(ph, fh, case.bc, case.length_xy, case.dzf, nthreads=os.cpu_count() or 1)
    assert res <= 1e-13, (res, info)
    assert np.isfinite(ph).all()
