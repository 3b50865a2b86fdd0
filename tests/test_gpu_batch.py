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
