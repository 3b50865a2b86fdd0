"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins notice each one.

Fault 1 uses the wrong z metric index in the stencil, fault 2 pairs each mode with its neighbour's
eigenvalue, fault 3 transposes the x basis on the way back; faults 4-8 (below) sit in the advection
term and the stable time step.  The correct oracle is restored after every case.
"""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I
from tests.test_oracle_pins import dense_operator, dense_solve, volumes

P, NN, DD = oracle.BC_P, oracle.BC_NN, oracle.BC_DD


def _lu_mismatch(bc=(P, DD, NN)):
    n = (8, 6, 8)
    dzf = I.tanh_dzf(8, 1.8)
    L = (1.0, 1.0)
    f = np.random.default_rng(11).uniform(-1, 1, (8, 6, 8))
    ref = dense_solve(dense_operator(n, bc, L, dzf), f.ravel()).reshape(f.shape)
    p = oracle.poisson_solve(f, bc, L, dzf)
    return np.linalg.norm(p - ref) / np.linalg.norm(ref)


def _manufactured_mismatch(bc=(P, DD, NN)):
    dzf = I.tanh_dzf(8, 1.8)
    p0 = np.random.default_rng(12).standard_normal((8, 6, 8))
    f = oracle.apply_laplacian(p0, bc, (1.0, 1.0), dzf)
    return np.linalg.norm(oracle.poisson_solve(f, bc, (1.0, 1.0), dzf) - p0) / np.linalg.norm(p0)


def _stencil_eigen_mismatch(bc=NN, n=8):
    A = dense_operator((n, 1, 1), (bc, P, NN), (float(n), 1.0), np.ones(1))
    E, lam = oracle.eigenbasis(bc, n)
    return np.abs(A @ E - E * lam[None, :]).max()


@pytest.fixture
def faulty():
    def plant(mode):
        oracle.set_fault(mode)

    yield plant
    oracle.set_fault(0)


def test_correct_oracle_passes_all_checks():
    assert _lu_mismatch() < 1e-12
    assert _manufactured_mismatch() < 1e-12
    assert _stencil_eigen_mismatch() < 1e-12


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_planted_mistake_is_caught(faulty, mode):
    faulty(mode)
    caught = (_lu_mismatch() > 1e-6) or (_manufactured_mismatch() > 1e-6) or (_stencil_eigen_mismatch() > 1e-6)
    assert caught, f"fault {mode} slipped through the pins"


# Faults 4-8 sit in the fractional-step pieces: 4 and 5 swap the z metric of the advection term's
# z-flux divergence (u: cell width -> centre distance; w: the reverse), 6 puts the cell width in the
# z row of the inverse time scale, 7 averages the wrong pair of w faces in its x row, 8 divides the
# y row's v term by the x spacing.
from tests.test_oracle_rk3_pins import _continuum_advection, advection_orders, dt_mismatches  # noqa: E402


def test_correct_oracle_passes_the_step_pins():
    orders, _ = advection_orders()
    assert (orders > 1.75).all()
    assert max(dt_mismatches().values()) < 1e-14


@pytest.mark.parametrize("mode", [4, 5, 6, 7, 8])
def test_planted_step_mistake_is_caught(faulty, mode):
    fields = _continuum_advection()
    faulty(mode)
    orders, _ = advection_orders(fields)
    caught = (orders < 1.75).any() or max(dt_mismatches().values()) > 1e-6
    assert caught, f"fault {mode} slipped through the pins"
