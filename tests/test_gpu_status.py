"""The plan's device status word (cans_plan_status): errors a solve detects on the device surface
without `info`, including from solves replayed out of a CUDA graph, and ordinary solves leave it
clear.

Failures are made on the host side of the inputs only (a right-hand side with a mean on a singular
problem, a tolerance no refinement can reach, a NaN in f), or, for the bounded device-side waits, by a
transaction barrier whose announced bytes no copy delivers; nothing here faults or hangs the GPU.
"""
import numpy as np
import pytest

from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN, DD = 0, 1, 2
OK, INCOMPATIBLE, NOT_CONVERGED, TIMEOUT = 0, -5, -6, -7


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def _rhs(n, bc, dzf, offset=0.0):
    """U[-1, 1] with its dzf-weighted mean removed (compatible), plus a constant offset."""
    case = I.case_uniform32(n=n)
    case.bc, case.dzf = bc, dzf
    return I.rhs_host(case) + offset


def _graph_replay(solver, f, p, reps=2):
    import torch

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        solver.solve(f, p, stream=s)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    solver.status()  # start from a clear word
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        solver.solve(f, p, stream=torch.cuda.current_stream())
    for _ in range(reps):
        g.replay()
    torch.cuda.synchronize()
    return g


CASES = [
    ((32, 24, 16), (P, P, NN), "tanh"),
    ((32, 24, 16), (P, DD, NN), "tanh"),
    ((32, 24, 16), (NN, NN, NN), "uniform"),
    ((32, 24, 16), (P, P, P), "uniform"),
    ((256, 128, 12), (P, P, NN), "tanh"),  # warp-engine x / y kernels and the streaming residual
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,bc,z", CASES)
def test_ordinary_solves_leave_the_word_clear(cans, prec, n, bc, z):
    import torch

    dzf = I.tanh_dzf(n[2], 1.6) if z == "tanh" else I.uniform_dzf(n[2])
    f = torch.from_numpy(_rhs(n, bc, dzf)).cuda()
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=prec, sweeps=2, verify=True)
    p = torch.empty_like(f)
    for _ in range(2):
        s.solve(f, p)
    assert s.status() == OK
    _graph_replay(s, f, p)
    assert s.status() == OK
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("bc,z", [((P, P, NN), "tanh"), ((P, P, P), "uniform"), ((NN, P, NN), "uniform")])
def test_incompatible_rhs_surfaces_from_graph_replay(cans, prec, bc, z):
    import torch

    n = (32, 24, 16)
    dzf = I.tanh_dzf(n[2], 1.6) if z == "tanh" else I.uniform_dzf(n[2])
    f = torch.from_numpy(_rhs(n, bc, dzf, offset=0.3)).cuda()
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=prec, sweeps=2)
    p = torch.empty_like(f)
    _graph_replay(s, f, p)
    assert s.status() == INCOMPATIBLE
    assert s.status() == OK  # reading clears the word
    # a tiny mean, far below the threshold, is not flagged
    f2 = torch.from_numpy(_rhs(n, bc, dzf, offset=1e-13)).cuda()
    s.solve(f2, p)
    assert s.status() == OK
    # a Helmholtz shift makes the problem non-singular: no compatibility condition
    s.solve(f, p, shift=-10.0)
    assert s.status() == OK
    s.close()


def test_unreachable_tolerance_surfaces_with_verify(cans):
    import torch

    n, bc = (64, 48, 20), (P, DD, NN)
    dzf = I.tanh_dzf(n[2], 1.8)
    f = torch.from_numpy(_rhs(n, bc, dzf)).cuda()
    p = torch.empty_like(f)
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=1, tol=1e-20, verify=True)
    _graph_replay(s, f, p)
    assert s.status() == NOT_CONVERGED
    s.close()
    # the same tolerance without verify: one sweep gives no stall to see, so the word stays clear
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=1, tol=1e-20)
    _graph_replay(s, f, p)
    assert s.status() == OK
    s.close()


def test_stalled_refinement_is_flagged_without_verify(cans):
    """Six sweeps reach the FP64 floor after two; from there a sweep no longer halves the residual.
    That stall is an error only while the residual is above tol."""
    import torch

    n, bc = (64, 48, 20), (P, DD, NN)
    dzf = I.tanh_dzf(n[2], 1.8)
    f = torch.from_numpy(_rhs(n, bc, dzf)).cuda()
    p = torch.empty_like(f)
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=6, tol=1e-20)
    _graph_replay(s, f, p)
    assert s.status() == NOT_CONVERGED
    s.close()
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=6, tol=1e-12)
    _graph_replay(s, f, p)
    assert s.status() == OK
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_non_finite_rhs_is_flagged(cans, prec):
    import torch

    n, bc = (32, 24, 16), (P, DD, NN)
    dzf = I.tanh_dzf(n[2], 1.6)
    fh = _rhs(n, bc, dzf)
    fh[3, 5, 7] = np.nan
    f = torch.from_numpy(fh).cuda()
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=prec, sweeps=2)
    p = torch.empty_like(f)
    s.solve(f, p)
    assert s.status() == NOT_CONVERGED
    s.close()


def test_info_call_returns_and_clears_the_word(cans):
    import torch

    n, bc = (32, 24, 16), (P, P, NN)
    dzf = I.tanh_dzf(n[2], 1.6)
    f = torch.from_numpy(_rhs(n, bc, dzf, offset=0.3)).cuda()
    g = torch.from_numpy(_rhs(n, bc, dzf)).cuda()
    s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=2)
    p = torch.empty_like(f)
    s.solve(f, p)  # records INCOMPATIBLE, no info
    _, info, st = s.solve(g, p, info=True)  # a compatible solve with info returns the recorded error
    assert st == INCOMPATIBLE
    assert s.status() == OK
    _, info, st = s.solve(g, p, info=True)
    assert st == OK and info[-1] <= 1e-12
    s.close()


def test_batched_device_status_flags_unreached_tolerance(cans):
    import torch

    n, bc = (48, 32, 12), (P, DD, NN)
    dzf = I.tanh_dzf(n[2], 1.6)
    plans, fs, ps, solvers = [], [], [], []
    for tol in (1e-12, 1e-20, 1e-12):
        s = cans.PoissonSolver(n, bc, (1.0, 1.0), dzf, prec=1, sweeps=1, tol=tol, verify=True)
        solvers.append(s)
        plans.append(s.plan)
        fs.append(torch.from_numpy(_rhs(n, bc, dzf)).cuda())
        ps.append(torch.empty_like(fs[-1]))
    status = torch.full((3,), 99, dtype=torch.int32, device="cuda")
    nbytes = cans.cans_poisson_batched_workspace_size(plans)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    st = cans.cans_poisson_solve_batched(plans, [t.data_ptr() for t in fs], [t.data_ptr() for t in ps],
                                         ws.data_ptr() + off, int(torch.cuda.current_stream().cuda_stream),
                                         status.data_ptr())
    torch.cuda.synchronize()
    assert st == 0
    assert status.cpu().tolist() == [OK, NOT_CONVERGED, OK]
    for s in solvers:
        s.close()


@pytest.mark.parametrize("graph", [False, True])
def test_bounded_wait_that_runs_out_records_timeout(cans, graph):
    """The bounded wait of the TMA-fed z kernels on a barrier that never completes (16 bytes announced,
    none delivered, no copy in flight) gives up after its polls and leaves CANS_ERR_TIMEOUT in the
    plan's status word -- also from a graph replay; a barrier that completes leaves the word clear."""
    import torch

    n = (32, 24, 16)
    s = cans.PoissonSolver(n, (P, P, NN), (1.0, 1.0), I.tanh_dzf(16, 1.5), prec=1)
    assert s.status() == OK
    cans.cans_check_bounded_wait(s.plan, 200, complete=True)
    assert s.status() == OK
    if graph:
        st = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            cans.cans_check_bounded_wait(s.plan, 200, complete=False, stream=st)
        assert s.status() == OK  # capture launches nothing
        g.replay()
    else:
        cans.cans_check_bounded_wait(s.plan, 200, complete=False)
    torch.cuda.synchronize()
    assert s.status() == TIMEOUT
    assert s.status() == OK  # read and cleared
    # the plan still solves after a recorded timeout
    f = torch.from_numpy(_rhs(n, (P, P, NN), I.tanh_dzf(16, 1.5))).cuda()
    s.solve(f)
    assert s.status() == OK
    s.close()
