"""Work partitioning across ranks (one process per GPU).

Circuits, and within a circuit the variants, are independent units, so a
multi-GPU run gives each rank a contiguous share of the units and needs no
collective on the data path; only the step time is reduced (max over ranks).
The contraction over the 4^k cut index can also be split: each rank sums a
contiguous range of cut terms and one sum-reduction of the 2^|o| partial
marginal combines them (the only exchange the method has).
"""
from __future__ import annotations


def shard_range(n_units: int, rank: int, world: int):
    """Contiguous [lo, hi) share of n_units for `rank` (sizes differ by <= 1)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_items(items, rank: int, world: int):
    lo, hi = shard_range(len(items), rank, world)
    return items[lo:hi]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank time (the step time of a weak-scaling run)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(array, dist=None, device=None):
    """Sum-reduce a partial result (e.g. a split-K partial marginal)."""
    import torch
    t = torch.as_tensor(array, dtype=torch.float64, device=device).clone()
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
