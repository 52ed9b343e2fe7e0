"""Host-side sharding of the FCA EM across processes (one GPU each).

Every quantity of the EM is indexed by the frequency bin and the likelihood of Eq. (like)
factorises over bins, so a mixture splits into contiguous bin ranges that run with no
exchange at all; the only cross-rank reduction is the sum of the per-iteration
log-likelihoods (and, for reporting, the max of the timed regions). Independent mixtures
shard trivially (one or more per rank).
"""
from __future__ import annotations


def frequency_shard(F: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced range [lo, hi) of the F bins owned by `rank` of `world`."""
    if world < 1 or not 0 <= rank < world or F < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(F, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def mixture_shard(n_mixtures: int, rank: int, world: int) -> list[int]:
    """Mixture indices owned by `rank` (round robin)."""
    return list(range(rank, n_mixtures, world))


def allreduce_sum(values, dist, device=None):
    """Sum of a float64 vector over ranks (the log-likelihood of Eq. (like) summed over all
    bins). `dist` is torch.distributed with an initialised process group."""
    import torch
    t = torch.as_tensor(values, dtype=torch.float64, device=device).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def allreduce_max(x: float, dist, device=None) -> float:
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, world: int, slowest_seconds: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / slowest_seconds
