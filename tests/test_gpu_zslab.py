"""The z-slab split of one solve (cans_zslab_*), emulated on one GPU: P ranks' slabs go through the
same kernels in one process, the exchange being a concatenation; the assembled solution must equal
the single-GPU FP64 solve and the oracle (Eq. poi_reduced) to FP64 accuracy, for singular and
non-singular problems, stretched z, uneven slabs and one-plane slabs.  (On several GPUs the exchange
is torch.distributed's all-gather; its host side is covered by the gloo test.)"""
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


@pytest.mark.parametrize(
    "n,bc,nranks",
    [((32, 24, 40), (P, P, NN), 2), ((48, 32, 33), (P, DD, NN), 3), ((16, 16, 9), (NN, DD, DD), 4),
     ((16, 8, 5), (P, P, NN), 5), ((64, 48, 64), (NN, P, NN), 1), ((256, 64, 96), (P, P, NN), 8)],
)
def test_zslab_emulated_ranks_match_single_gpu_solve(cans, n, bc, nranks):
    import torch

    from paper_2001_05234_b300.zslab import ZSlabSolver

    dzf = I.tanh_dzf(n[2], 1.7)
    case = I.case_uniform32(n=n)
    case.bc, case.dzf = bc, dzf
    f = I.rhs_host(case)
    ft = torch.from_numpy(f).cuda()
    solvers = [ZSlabSolver(n, bc, (1.0, 0.8), dzf, nranks, r) for r in range(nranks)]
    outs, ifs, cols = [], [], []
    for s in solvers:
        slab = ft[s.z0:s.z1].contiguous()
        out = torch.empty_like(slab)
        iface, col00 = s.eliminate(slab, out)
        outs.append(out)
        ifs.append(iface)
        cols.append(col00)
    iface_all, col00_all = torch.cat(ifs), torch.cat(cols)
    for s, out in zip(solvers, outs):
        s.finish(out, iface_all, col00_all)
    got = torch.cat(outs).cpu().numpy()
    one = cans.PoissonSolver(n, bc, (1.0, 0.8), dzf, prec=0)
    ref_gpu = one.solve(ft).cpu().numpy()
    one.close()
    ref = oracle.poisson_solve(f, bc, (1.0, 0.8), dzf)
    assert np.linalg.norm(got - ref_gpu) <= 1e-12 * np.linalg.norm(ref_gpu)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    for s in solvers:
        s.close()


def test_zslab_rejects_periodic_and_mixed_plans(cans):
    o = cans.cans_opts_default()
    _, h = cans.cans_poisson_plan((16, 16, 8), (1.0, 1.0), (P, P, P), None, o)
    with pytest.raises(cans.CansError):
        cans.cans_zslab_create(h, 0, 4)
    cans.cans_plan_destroy(h)
    o.prec = 1
    _, h = cans.cans_poisson_plan((16, 16, 8), (1.0, 1.0), (P, P, NN), None, o)
    with pytest.raises(cans.CansError):
        cans.cans_zslab_create(h, 0, 4)
    cans.cans_plan_destroy(h)
