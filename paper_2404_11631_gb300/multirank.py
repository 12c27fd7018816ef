"""Host-side logic for runs over several ranks (one process per GPU).

Independent instances per rank (the weak-scaling layout the benchmark uses):
rank r evaluates instance r of the workload, and the whole-job figure is the
total work over the slowest rank's time.  No collective touches the data
path; the only collective is the max of the ranks' times.

Splitting ONE instance's N scenarios across R ranks would need one exchange:
each rank holds the FP64 partial sums of its scenario range (S1, S2 per
decision, m~ per dimension, G per decision and dimension), one all-reduce
adds them, and every rank finalizes (Eq. 4 and its gradient) from the
totals.  ``scenario_ranges`` and ``merge_partials`` give that exchange; the
tests run it over gloo on the CPU.
"""
from __future__ import annotations


def instance_for_rank(rank: int) -> int:
    """Instance id (Philox counter word 3) of rank ``rank`` in weak scaling."""
    return int(rank)


def scenario_ranges(N: int, world: int) -> list[tuple[int, int]]:
    """Contiguous scenario ranges [a, b) of N scenarios over ``world`` ranks."""
    return [(N * r // world, N * (r + 1) // world) for r in range(world)]


def max_time_over_ranks(seconds: float) -> float:
    """Slowest rank's time (requires an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def merge_partials(partials):
    """Sum of the ranks' FP64 partial vectors with one all-reduce (in place
    on a CPU float64 tensor; returns the totals)."""
    import torch
    import torch.distributed as dist
    t = partials.to(torch.float64).clone()
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
