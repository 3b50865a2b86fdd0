"""The adjoint of the Poisson solve (cans_poisson_solve_adjoint): <S f, g> = <f, S^T g> for random f, g
(compatible or not: S projects), stretched z, singular and regular boundary combinations, FP64 and
mixed precision; the torch autograd wrapper's gradient against central differences."""
import numpy as np
import pytest

from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD = 0, 1, 2


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("bc", [(P, P, NN), (P, DD, NN), (NN, NN, DD), (DD, P, NN), (P, P, P)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-11)])
def test_dot_product_identity(cans, bc, prec, tol):
    n = (48, 32, 24)
    dzf = I.tanh_dzf(24, 1.7, 1.3) if bc[2] != P else I.uniform_dzf(24)
    s = cans.PoissonSolver(n, bc, (1.2, 0.9), dzf, prec=prec, sweeps=2)
    rng = np.random.default_rng(31)
    fh = rng.standard_normal((24, 32, 48))
    if all(b != DD for b in bc):  # singular: a compatible f (zero dzf-weighted mean), as a divergence is
        fh -= (fh * dzf[:, None, None]).sum() / (dzf.sum() * 32 * 48)
    f = dev(fh)
    g = dev(rng.standard_normal((24, 32, 48)))  # g arbitrary: the adjoint projects it
    sf = s.solve(f)
    stg = s.solve_adjoint(g)
    lhs = float((sf * g).sum())
    rhs = float((f * stg).sum())
    assert abs(lhs - rhs) <= tol * max(abs(lhs), 1e-30) * 10, (lhs, rhs)
    s.close()


def test_adjoint_in_place_and_uniform_self_adjoint(cans):
    import torch

    n = (32, 16, 16)
    s = cans.PoissonSolver(n, (P, NN, NN), (1.0, 1.0), I.uniform_dzf(16))
    g = dev(np.random.default_rng(2).standard_normal((16, 16, 32)))
    want = s.solve(g)  # uniform grid: S is symmetric, S^T g = S g
    q = g.clone()
    s.solve_adjoint(q, out=q)
    torch.cuda.synchronize()
    assert float((q - want).abs().max()) <= 1e-12 * float(want.abs().max())
    s.close()


def test_autograd_gradient_matches_finite_differences(cans):
    import torch

    n = (16, 16, 16)
    dzf = I.tanh_dzf(16, 1.8, 1.0)
    s = cans.PoissonSolver(n, (P, DD, NN), (1.0, 1.0), dzf)
    rng = np.random.default_rng(8)
    f0 = dev(rng.standard_normal((16, 16, 16)))
    wgt = dev(rng.standard_normal((16, 16, 16)))

    def loss(f):
        return (cans.poisson_solve(s, f) * wgt).sum()

    x = f0.clone().requires_grad_(True)
    loss(x).backward()
    grad = x.grad.detach()
    for d in range(6):
        e = dev(rng.standard_normal((16, 16, 16)))
        h = 1e-6 * float(torch.linalg.vector_norm(f0))
        with torch.no_grad():
            fd = float((loss(f0 + h * e) - loss(f0 - h * e)) / (2 * h))
        ad = float((grad * e).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (d, fd, ad)
    s.close()
