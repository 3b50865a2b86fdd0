"""Batched ensemble of uneven problems (cans_batch_*): every problem matches its own single solve and
the FP64 oracle; the batch replays inside a CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_2001_05234_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cans():
    from paper_2001_05234_b300 import build_lib

    build_lib.build()
    import paper_2001_05234_b300 as C

    return C


def test_batch_matches_single_solves_and_oracle(cans):
    import torch

    cases = I.ensemble_cases(count=12, sizes=(16, 24, 32, 48))
    fs = [torch.from_numpy(I.rhs_host(c)).cuda() for c in cases]
    ps = [torch.full_like(f, float("nan")) for f in fs]
    b = cans.Batch(cases, prec=cans.CANS_MIXED, sweeps=2, nstreams=4)
    b.solve(fs, ps)
    torch.cuda.synchronize()
    for c, f, p in zip(cases, fs, ps):
        ref = oracle.poisson_solve(f.cpu().numpy(), c.bc, c.length_xy, c.dzf)
        got = p.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-11, (c.n, c.bc, err)
        res = oracle.relative_residual(got, f.cpu().numpy(), c.bc, c.length_xy, c.dzf)
        floor = oracle.relative_residual(ref, f.cpu().numpy(), c.bc, c.length_xy, c.dzf)
        assert res <= max(1e-12, 2 * floor), (c.n, c.bc, res, floor)
    b.close()


def test_batch_in_cuda_graph(cans):
    import torch

    cases = I.ensemble_cases(count=8, sizes=(32, 48, 64))
    fs = [torch.from_numpy(I.rhs_host(c)).cuda() for c in cases]
    eager = [torch.empty_like(f) for f in fs]
    b = cans.Batch(cases, prec=cans.CANS_MIXED, sweeps=2, nstreams=4)
    b.solve(fs, eager)
    torch.cuda.synchronize()
    out = [torch.empty_like(f) for f in fs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.solve(fs, out)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for a, e in zip(out, eager):
        assert float((a - e).abs().max()) <= 1e-13 * float(e.abs().max())
    b.close()


@pytest.mark.slow
def test_full_ensemble_64_problems(cans):
    """The 64-problem ensemble (dims from {32, ..., 192}): per-problem error vs the FP64 oracle on a sample."""
    import torch

    cases = I.ensemble_cases()
    fs = [torch.from_numpy(I.rhs_host(c)).cuda() for c in cases]
    ps = [torch.empty_like(f) for f in fs]
    b = cans.Batch(cases, prec=cans.CANS_MIXED, sweeps=2)
    b.solve(fs, ps)
    torch.cuda.synchronize()
    small = sorted(range(len(cases)), key=lambda q: cases[q].points)[:6]
    for q in small:
        c = cases[q]
        ref = oracle.poisson_solve(fs[q].cpu().numpy(), c.bc, c.length_xy, c.dzf)
        err = np.linalg.norm(ps[q].cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-11, (c.n, c.bc, err)
    for q in range(len(cases)):  # every problem: residual via the oracle's operator
        c = cases[q]
        res = oracle.relative_residual(ps[q].cpu().numpy(), fs[q].cpu().numpy(), c.bc, c.length_xy, c.dzf)
        assert res <= 1e-11, (c.n, c.bc, res)
    b.close()


def test_solve_batched_one_call_with_status(cans):
    """cans_poisson_solve_batched: the one-call form writes the same results as the batch object and
    a zero status per problem; a workspace that is not 256-byte aligned is refused before any launch."""
    import torch

    cases = I.ensemble_cases(count=6, sizes=(16, 32, 48))
    fs = [torch.from_numpy(I.rhs_host(c)).cuda() for c in cases]
    ref = [torch.empty_like(f) for f in fs]
    b = cans.Batch(cases, prec=cans.CANS_MIXED, sweeps=2, nstreams=8)
    b.solve(fs, ref)
    torch.cuda.synchronize()
    nbytes = cans.cans_poisson_batched_workspace_size(b.plans)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    status = torch.full((len(cases),), -7, dtype=torch.int32, device="cuda")
    out = [torch.full_like(f, float("nan")) for f in fs]
    stream = torch.cuda.current_stream().cuda_stream
    rc = cans.cans_poisson_solve_batched(b.plans, [t.data_ptr() for t in fs], [t.data_ptr() for t in out], base,
                                         stream, status.data_ptr())
    torch.cuda.synchronize()
    assert rc == 0
    assert status.cpu().tolist() == [0] * len(cases)
    for a, e in zip(out, ref):
        assert float((a - e).abs().max()) <= 1e-13 * float(e.abs().max())
    rc = cans.cans_poisson_solve_batched(b.plans, [t.data_ptr() for t in fs], [t.data_ptr() for t in out], base + 8,
                                         stream, status.data_ptr())
    torch.cuda.synchronize()
    assert rc == cans.CANS_ERR_WORKSPACE
    assert status.cpu().tolist() == [rc] * len(cases)
    b.close()


def test_solve_batched_device_status_flags_nonfinite(cans):
    """A problem whose right-hand side holds a NaN is flagged CANS_ERR_NOT_CONVERGED in the device status
    of the one-call batched solve; its neighbours in the batch are unaffected and report CANS_OK."""
    import torch

    cases = I.ensemble_cases(count=4, sizes=(16, 32))
    fs = [torch.from_numpy(I.rhs_host(c)).cuda() for c in cases]
    fs[2].view(-1)[5] = float("nan")
    b = cans.Batch(cases, prec=cans.CANS_MIXED, sweeps=1, nstreams=4)
    ref = [torch.empty_like(f) for f in fs]
    b.solve(fs, ref)
    torch.cuda.synchronize()
    nbytes = cans.cans_poisson_batched_workspace_size(b.plans)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    status = torch.full((len(cases),), 99, dtype=torch.int32, device="cuda")
    out = [torch.empty_like(f) for f in fs]
    rc = cans.cans_poisson_solve_batched(b.plans, [t.data_ptr() for t in fs], [t.data_ptr() for t in out], base,
                                         torch.cuda.current_stream().cuda_stream, status.data_ptr())
    torch.cuda.synchronize()
    assert rc == 0
    assert status.cpu().tolist() == [0, 0, -6, 0]
    for q in (0, 1, 3):
        assert float((out[q] - ref[q]).abs().max()) <= 1e-13 * float(ref[q].abs().max())
    b.close()


def test_solve_batched_one_call_replays_from_a_graph(cans):
    """The one-call batched solve takes its internal streams from a per-device pool created by the first
    call, so a later call can be captured into a CUDA graph; replays give the eager results and the
    per-problem status."""
    import torch

    cases = I.ensemble_cases(count=5, sizes=(16, 32, 48))
    fs = [torch.from_numpy(I.rhs_host(c)).cuda() for c in cases]
    b = cans.Batch(cases, prec=cans.CANS_MIXED, sweeps=2, nstreams=4)
    nbytes = cans.cans_poisson_batched_workspace_size(b.plans)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    status = torch.full((len(cases),), 99, dtype=torch.int32, device="cuda")
    ref = [torch.empty_like(f) for f in fs]
    out = [torch.full_like(f, float("nan")) for f in fs]
    # eager first (creates the pool outside any capture)
    assert cans.cans_poisson_solve_batched(b.plans, [t.data_ptr() for t in fs], [t.data_ptr() for t in ref], base,
                                           torch.cuda.current_stream().cuda_stream, status.data_ptr()) == 0
    torch.cuda.synchronize()
    status.fill_(99)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        rc = cans.cans_poisson_solve_batched(b.plans, [t.data_ptr() for t in fs], [t.data_ptr() for t in out], base,
                                             s.cuda_stream, status.data_ptr())
    assert rc == 0
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * len(cases)
    for a, e in zip(out, ref):
        assert torch.equal(a, e)
    b.close()
