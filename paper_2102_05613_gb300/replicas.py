"""Replicas across GPUs: chains and disorder instances are independent, so
each rank runs its own chains with its own seeds (weak scaling) and there is
no exchange on the sampling path.  The only collectives are the reductions
of timings and of FP64 observable sums at the end.
"""
from __future__ import annotations


def seed_base(rank: int) -> int:
    """Coupling and chain seeds of rank r start at 1000 r (disjoint per rank)."""
    return 1000 * int(rank)


def _tensor(x, device):
    import torch
    return torch.tensor([float(x)], dtype=torch.float64, device=device)


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest `value` over ranks (the job's wall time is the slowest rank's)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    t = _tensor(value, device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(values, dist=None, device="cpu"):
    """Element-wise FP64 sums over ranks (e.g. observable sums and counts)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]
