"""Runs over several ranks (one process per GPU).

Two layouts:

* Independent instances (the benchmark's weak scaling): rank r evaluates
  instance r of the workload (Philox counter word 3), no collective touches
  the data path, and the whole-job figure is the total work over the slowest
  rank's time (``max_time_over_ranks``).

* One problem's N samples split across the ranks (the sums over i in Eq. 4
  and Eq. 5 of Sec. 3.1 are sums of independent terms, and the counter-based
  generator lets rank r draw exactly its own scenarios): rank r takes the
  contiguous range ``scenario_ranges(N, R)[r]``, ``saa_partials`` writes the
  range's FP64 partial sums [P1 | P2 | P3 | P4] on its GPU, one collective
  adds them (``merge_partials``: an all-reduce of 2K + d (+ K d) doubles, the
  only exchange of the method), and every rank finalizes Eq. 4, Eq. 5 and
  the gradient from the totals with ``saa_finalize_partials``
  (``estimate_sharded``).  The merge is either the collective's own sum
  (``ordered=False``) or an all-gather followed by a sum in rank order, which
  gives the same totals bit for bit whatever the collective's reduction
  order is.
"""
from __future__ import annotations


def instance_for_rank(rank: int) -> int:
    """Instance id (Philox counter word 3) of rank ``rank`` in weak scaling."""
    return int(rank)


def scenario_ranges(N: int, world: int) -> list[tuple[int, int]]:
    """Contiguous scenario ranges [a, b) of N scenarios over ``world`` ranks
    (sizes differ by at most one; every range is non-empty when N >= world)."""
    if world < 1 or N < world:
        raise ValueError("need 1 <= world <= N")
    return [(N * r // world, N * (r + 1) // world) for r in range(world)]


def _group():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized()


def max_time_over_ranks(seconds: float) -> float:
    """Slowest rank's time (1 rank without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not _group():
        return float(seconds)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def merge_partials(part, ordered: bool = True):
    """Totals of the ranks' partial vectors (same length on every rank).

    ordered=True (CUDA tensors) gathers every rank's vector and adds them in
    rank order with libsaa's saa_partials_merge, so the totals do not depend
    on how the collective schedules its reduction; ordered=False uses one
    all-reduce (its sum).  Returns a new float64 tensor on the input's
    device; without a process group, the input's values."""
    import torch
    import torch.distributed as dist
    t = part.to(torch.float64).contiguous()
    if not _group():
        return t.clone()
    if not ordered or not t.is_cuda:
        t = t.clone()
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t
    from . import saa
    rows = torch.empty(dist.get_world_size(), t.numel(), dtype=torch.float64, device=t.device)
    dist.all_gather_into_tensor(rows, t)
    return saa.saa_partials_merge(rows)


def estimate_sharded(prob, X, prec="fp32", grad: bool = False, ordered: bool = True) -> dict:
    """Eq. 4, Eq. 5 (and the gradient) of one problem whose N samples are
    split across the ranks of the process group (or all on this GPU without
    one): this rank's range through saa_partials, the merge, then
    saa_finalize_partials on every rank."""
    import torch.distributed as dist

    from . import saa
    rank, world = (dist.get_rank(), dist.get_world_size()) if _group() else (0, 1)
    a, b = scenario_ranges(int(prob.N), world)[rank]
    part = saa.saa_partials(prob, a, b - a, X, prec, grad=grad)
    tot = merge_partials(part, ordered=ordered)
    return saa.saa_finalize_partials(prob, X, tot, grad=grad)
