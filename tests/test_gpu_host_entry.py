"""cans_poisson_solve_host: the solve from and to host memory in one C-ABI call (upload on a copy-in
stream, the solve on a compute stream, the download on a copy-out stream, ordered by the plan's
events).  Its result equals the device-to-device solve of the same plan bit for bit, on one stream and
on three; pipelined calls with alternating device buffers (the loop bench.py times) give each step its
own right-hand side's solution; the three streams captured into one CUDA graph replay correctly;
pageable host memory works (synchronously) as well; bad arguments are refused before anything is
enqueued."""
import numpy as np
import pytest

from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu

P, NN = 0, 1


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("streams", [1, 3])
def test_host_solve_equals_device_solve(cans, prec, streams):
    import torch

    n = (256, 64, 40)
    case = I.case_modes(n=n)
    case.length_xy = (256 / 1024, 64 / 1024)
    case.dzf = I.tanh_dzf(40, 1.6)
    f = I.rhs_host(case)
    s = cans.PoissonSolver(n, case.bc, case.length_xy, case.dzf, prec=prec, sweeps=2)
    ft = torch.from_numpy(f).cuda()
    want = s.solve(ft).cpu().numpy()
    fh = torch.from_numpy(f).pin_memory()
    ph = torch.full_like(fh, np.nan).pin_memory()
    fd, pd = torch.empty_like(ft), torch.empty_like(ft)
    st = [torch.cuda.Stream() for _ in range(streams)]
    s.solve_host(fh, ph, fd, pd, copy_in=st[0], compute=st[-1 if streams == 1 else 1], copy_out=st[-1])
    torch.cuda.synchronize()
    assert np.array_equal(ph.numpy(), want)
    s.close()


def test_pipelined_host_solves_keep_each_step_apart(cans):
    """Four steps with different right-hand sides through alternating device buffers on three streams,
    guarded as bench.py guards them: every step's host output is its own solution."""
    import torch

    n = (128, 32, 24)
    dzf = I.tanh_dzf(24, 1.5)
    s = cans.PoissonSolver(n, (P, P, NN), (1.0, 1.0), dzf, prec=1, sweeps=2)
    fs = [I.rhs_host(I.PoissonCase("h", n, (P, P, NN), (1.0, 1.0), dzf, 4280 + k, "uniform")) for k in range(4)]
    want = [s.solve(torch.from_numpy(f).cuda()).cpu().numpy() for f in fs]
    fh = [torch.from_numpy(f).pin_memory() for f in fs]
    ph = [torch.empty_like(fh[0]).pin_memory() for _ in range(4)]
    fd = [torch.empty(fs[0].shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    pd = [torch.empty_like(fd[0]) for _ in range(2)]
    s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    done, out = [torch.cuda.Event() for _ in range(4)], [torch.cuda.Event() for _ in range(4)]
    for k in range(4):
        b = k % 2
        if k >= 2:
            s_in.wait_event(done[k - 2])
            s_c.wait_event(out[k - 2])
        s.solve_host(fh[k], ph[k], fd[b], pd[b], copy_in=s_in, compute=s_c, copy_out=s_out)
        done[k].record(s_c)
        out[k].record(s_out)
    torch.cuda.synchronize()
    for k in range(4):
        assert np.array_equal(ph[k].numpy(), want[k])
    s.close()


def test_pageable_host_memory_and_argument_checks(cans):
    import torch

    n = (64, 32, 16)
    dzf = I.tanh_dzf(16, 1.5)
    s = cans.PoissonSolver(n, (P, P, NN), (1.0, 1.0), dzf, prec=0)
    f = I.rhs_host(I.PoissonCase("h", n, (P, P, NN), (1.0, 1.0), dzf, 4290, "uniform"))
    want = s.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    fh, ph = torch.from_numpy(f.copy()), torch.zeros(f.shape, dtype=torch.float64)
    fd, pd = torch.empty(f.shape, dtype=torch.float64, device="cuda"), torch.empty(f.shape, dtype=torch.float64,
                                                                                    device="cuda")
    s.solve_host(fh, ph, fd, pd)
    torch.cuda.synchronize()
    assert np.array_equal(ph.numpy(), want)
    L = cans.lib()
    assert L.cans_poisson_solve_host(s.plan, fh.data_ptr(), ph.data_ptr(), fd.data_ptr(), fd.data_ptr(), None, None,
                                     None, None) == cans.CANS_ERR_ARG  # in place refused
    assert L.cans_poisson_solve_host(None, fh.data_ptr(), ph.data_ptr(), fd.data_ptr(), pd.data_ptr(), None, None,
                                     None, None) == cans.CANS_ERR_ARG
    s.close()
    sm = cans.PoissonSolver(n, (P, P, NN), (1.0, 1.0), dzf, prec=1)
    assert L.cans_poisson_solve_host(sm.plan, fh.data_ptr(), ph.data_ptr(), fd.data_ptr(), pd.data_ptr(), None, None,
                                     None, None) == cans.CANS_ERR_WORKSPACE  # mixed needs its workspace
    sm.close()



def test_host_solve_captured_in_a_cuda_graph(cans):
    """Upload, solve and download on three streams captured into one CUDA graph (the plan's events
    become the graph's edges); replays with a new right-hand side in the pinned input buffer give its
    solution."""
    import torch

    n = (128, 32, 24)
    dzf = I.tanh_dzf(24, 1.5)
    s = cans.PoissonSolver(n, (P, P, NN), (1.0, 1.0), dzf, prec=1, sweeps=2)
    fs = [I.rhs_host(I.PoissonCase("g", n, (P, P, NN), (1.0, 1.0), dzf, 4300 + k, "uniform")) for k in range(2)]
    want = [s.solve(torch.from_numpy(f).cuda()).cpu().numpy() for f in fs]
    fh = torch.from_numpy(fs[0].copy()).pin_memory()
    ph = torch.zeros_like(fh).pin_memory()
    fd = torch.empty(fs[0].shape, dtype=torch.float64, device="cuda")
    pd = torch.empty_like(fd)
    s.solve_host(fh, ph, fd, pd)  # warm-up outside the capture
    torch.cuda.synchronize()
    cap, s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        ev = torch.cuda.Event()
        ev.record(cap)
        s_in.wait_event(ev)  # fork the copy streams from the capture
        s_out.wait_event(ev)
        s.solve_host(fh, ph, fd, pd, copy_in=s_in, compute=cap, copy_out=s_out)
        done = torch.cuda.Event()
        done.record(s_out)
        cap.wait_event(done)  # join
    for k in range(2):
        fh.copy_(torch.from_numpy(fs[k]))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(ph.numpy(), want[k])
    s.close()
