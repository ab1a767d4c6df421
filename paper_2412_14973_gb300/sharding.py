"""Frequency sharding across GPUs (one process per GPU).

Frequencies are independent problems (the paper solves each frequency on its
own), so a multi-GPU run needs no collective on the data path: each rank
solves its own frequencies, only the timing is reduced (max over ranks), and
the per-frequency results are gathered on rank 0's host at the end.
"""
from __future__ import annotations


def shard(n: int, rank: int, world: int) -> list:
    """Frequencies of ``rank``: round-robin, so every rank gets a similar mix
    of low and high ranks (cost grows with the rank of the frequency)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    return list(range(rank, n, world))


def frequency_plan(n_per_gpu: int, rank: int, world: int) -> list:
    """Global frequency indices solved by ``rank`` when every GPU gets
    ``n_per_gpu`` frequencies (weak scaling): the job is one list of
    n_per_gpu * world frequencies with one rank schedule over all of them,
    dealt round-robin by shard()."""
    if n_per_gpu < 1:
        raise ValueError("n_per_gpu must be positive")
    return shard(n_per_gpu * world, rank, world)


def batches(freqs: list, batch: int) -> list:
    """Split a rank's frequencies into steps of ``batch``: step b takes every
    nb-th frequency starting at the b-th (nb = len(freqs) // batch), so each
    step spans the whole rank range and all steps cost about the same."""
    if batch < 1 or len(freqs) % batch:
        raise ValueError("the frequency count must be a multiple of the batch")
    nb = len(freqs) // batch
    return [freqs[b::nb] for b in range(nb)]


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Maximum of ``x`` over the ranks of the default process group (x if none)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(records: list, dist=None):
    """Every rank's per-frequency records (small host objects: frequency
    index, rank, final misfit, iterations, status) on rank 0, sorted by
    frequency; None on the other ranks.  Without a process group the records
    themselves."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return sorted(records, key=lambda r: r["freq"])
    world = dist.get_world_size()
    out = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(records, out, dst=0)
    if dist.get_rank() != 0:
        return None
    return sorted((r for part in out for r in part), key=lambda r: r["freq"])
