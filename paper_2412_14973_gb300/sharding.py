"""Frequency sharding across GPUs (one process per GPU).

Frequencies are independent problems (the paper solves each frequency on its
own), so a multi-GPU run needs no collective on the data path: each rank
solves its own frequencies and only the timing is reduced (max over ranks).
"""
from __future__ import annotations


def shard(n: int, rank: int, world: int) -> list:
    """Frequencies of ``rank``: round-robin, so every rank gets a similar mix
    of low and high ranks (cost grows with the rank of the frequency)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    return list(range(rank, n, world))


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Maximum of ``x`` over the ranks of the default process group (x if none)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
