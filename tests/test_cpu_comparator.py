"""The fair CPU comparator bench.py times beside the oracle (scipy.fft transforms + a vectorised numpy
Thomas sweep) solves the same discrete problem as the oracle on every x/y boundary-condition
combination, stretched z, in the singular and the non-singular case."""
import itertools
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("bx,by,bz", list(itertools.product((I.BC_P, I.BC_NN, I.BC_DD), (I.BC_P, I.BC_NN, I.BC_DD),
                                                             (I.BC_NN, I.BC_DD))))
def test_cpu_fft_solve_matches_oracle(bx, by, bz):
    n = (12, 10, 9)
    dzf = I.uniform(11, (n[2],), 0.5, 1.5)  # an arbitrary, asymmetric z grid
    dzf /= dzf.sum()
    f = I.uniform(7 + bx + 3 * by + 9 * bz, (n[2], n[1], n[0]), -1.0, 1.0)
    bc = (bx, by, bz)
    if I.BC_DD not in bc:
        f = I.weighted_mean_removed(f, dzf)
    ref = oracle.poisson_solve(f, bc, (1.3, 0.7), dzf)
    got = bench.cpu_fft_solve(f, bc, (1.3, 0.7), dzf, workers=2)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
