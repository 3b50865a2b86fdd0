"""The no-allocation solve entry point (for callers that cannot allocate device memory).

Collected last on purpose: if it fails, a run that stops at the first failure has already run every
other test.  It compares cans_poisson_solve_noalloc, which takes its workspace from the library's
fixed scratch array, with cans_poisson_solve given a caller-allocated workspace, on two calls in a
row (with a solve of another problem through the same scratch between them), and checks that a
problem larger than the scratch array is refused.
"""
import numpy as np
import pytest

from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _plan(C, case, prec):
    o = C.cans_opts_default()
    o.prec, o.max_sweeps = prec, 2
    return C.cans_poisson_plan(case.n, case.length_xy, case.bc, case.dzf, o)[1]


@pytest.mark.parametrize("prec", [1, 0])
def test_noalloc_solve_matches_workspace_solve(prec):
    import torch

    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    case = I.case_modes(n=(128, 96, 64))  # mixed workspace 9.4 MB, inside the 48 MiB scratch
    f = torch.from_numpy(I.rhs_host(case)).cuda()
    h = _plan(C, case, prec)
    nbytes = C.cans_poisson_workspace_size(h)
    assert nbytes <= C.cans_noalloc_scratch_bytes()
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) // 256 * 256 if nbytes else 0
    s = int(torch.cuda.current_stream().cuda_stream)
    ref = torch.empty_like(f)
    assert C.cans_poisson_solve(h, f.data_ptr(), ref.data_ptr(), wp, s, None) == 0
    # a problem of another shape and boundary conditions, solved through the same scratch between the
    # compared calls, leaves different stale data in it: a solve that read a scratch word before
    # writing it would no longer match
    other = I.case_channel(n=(96, 64, 40))
    g = torch.from_numpy(I.rhs_host(other)).cuda()
    q = torch.empty_like(g)
    h2 = _plan(C, other, 1)
    for call in range(2):  # two calls in a row share the scratch array
        out = torch.full_like(f, float("nan"))
        assert C.cans_poisson_solve_noalloc(h, f.data_ptr(), out.data_ptr(), s, None) == 0
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
        assert err <= 1e-12, err
        if call == 0:
            assert C.cans_poisson_solve_noalloc(h2, g.data_ptr(), q.data_ptr(), s, None) == 0
    C.cans_plan_destroy(h2)
    C.cans_plan_destroy(h)


def test_noalloc_rejects_problems_larger_than_the_scratch():
    import torch

    import paper_2001_05234_b300 as C

    case = I.case_modes(n=(256, 256, 128))  # 8.4M points: 100 MB of mixed workspace
    h = _plan(C, case, 1)
    assert C.cans_poisson_workspace_size(h) > C.cans_noalloc_scratch_bytes()
    f = torch.zeros(case.shape, dtype=torch.float64, device="cuda")
    p = torch.zeros_like(f)
    st = C.cans_poisson_solve_noalloc(h, f.data_ptr(), p.data_ptr(), int(torch.cuda.current_stream().cuda_stream),
                                      None)
    assert st == -4  # CANS_ERR_WORKSPACE, nothing enqueued
    C.cans_plan_destroy(h)
