"""Partition of independent instances across ranks (one process per GPU).

Every instance (one subcarrier with its right-hand sides) is an independent
CG solve of Algorithm 1, so ranks share no data: each rank takes its own
block of instances and nothing is exchanged on the data path. The only
collective a multi-rank run needs is the maximum of the ranks' elapsed
times, which is what a throughput report divides by.
"""

from __future__ import annotations


def instance_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block [start, stop) of n_total instances owned by `rank`.

    Blocks differ in size by at most one instance and cover 0..n_total-1
    exactly once across ranks 0..world-1.
    """
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and n_total >= 0")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over all ranks of the default process group (the
    value itself without one). Timing only; not part of the data path."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
