"""Host-side logic for running the solver on several GPUs of one node.

A single Poisson solve does not shard without an all-to-all exchange, so multi-GPU runs are replicas
(each rank solves its own problem, weak scaling) or an ensemble of independent problems split across
ranks by greedy size balancing.  No collective touches the data path: ranks only meet at barriers and
in one max-reduction of their timings.
"""
from __future__ import annotations


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest value over all ranks (the slowest rank's time); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gpts(points_per_rank: int, ms_per_step: float, world: int) -> float:
    """Whole-job throughput: points solved by all ranks per second of the slowest rank, in Gpts/s."""
    return world * points_per_rank / (ms_per_step * 1e-3) / 1e9


def assign_problems(sizes, world: int):
    """Greedy balancing of independent problems over `world` ranks: largest first onto the least
    loaded rank.  Returns one list of problem indices per rank (each index exactly once)."""
    order = sorted(range(len(sizes)), key=lambda q: (-sizes[q], q))
    load = [0] * world
    out = [[] for _ in range(world)]
    for q in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(q)
        load[r] += sizes[q]
    for lst in out:
        lst.sort()
    return out
