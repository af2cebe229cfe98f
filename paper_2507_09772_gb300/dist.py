"""Host-side logic of multi-GPU runs (one process per GPU).

Two ways to use several GPUs:
* independent batches (weak scaling): each rank builds its own batch of
  molecules; the only collectives are the timing barrier and the max/sum
  reductions of the step time and of the work done;
* one batch split across ranks: rank r sets the library options
  part_index = r, part_count = world; its J and K are then partial sums, and
  one sum all-reduce gives every rank the full result.
"""
from __future__ import annotations


def batch_seed_base(rank: int) -> int:
    """Seed base of the batch a rank builds in weak-scaling runs."""
    return 1001 + 1000 * int(rank)


def partition_options(rank: int, world: int) -> dict:
    return {"part_count": int(world), "part_index": int(rank)}


def reduce_step_timing(dist, ms: float, units: float, device=None):
    """(max of ms over ranks, sum of units over ranks)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def sum_partials(dist, tensors):
    """In-place sum all-reduce of partial J/K tensors (the exchange step)."""
    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tensors
