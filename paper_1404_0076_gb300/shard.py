"""Host logic for running the evaluator on N ranks (one process per GPU).

Nets share no agent and their interactions are local (Sec. 2.1), so the
units of work (nets of a batch, requests of a stream) partition across ranks
with no exchange on the data path: every rank reduces its own share on its
own GPU, and only the timing and the counts are combined at the end (the
slowest rank's time, the sum of interactions).  A single net does not
partition; it runs as independent replicas.
"""
from __future__ import annotations


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s synthetic batch: every rank draws a batch of the
    same shape from its own seed (weak scaling)."""
    return base + 1000 * rank


def partition(n: int, rank: int, world: int) -> range:
    """Indices of the `n` units that rank `rank` of `world` owns: contiguous
    blocks whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    return range(start, start + q + (1 if rank < r else 0))


def combine(seconds: float, interactions: int, dist=None) -> tuple[float, int]:
    """(max seconds over ranks, sum of interactions over ranks).  `dist` is
    an initialised torch.distributed module, or None for one rank."""
    if dist is None:
        return seconds, interactions
    import torch
    t = torch.tensor([seconds], dtype=torch.float64)
    n = torch.tensor([interactions], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())
