"""Multi-GPU helpers: sharding by independent column blocks, and job timing over ranks.

The hybrid subalgebra S_Hy^p (and the parallel one, p = 1) makes the q = k/p column blocks independent
problems (Section 3: the hybrid method is a data-parallel version of the classical method), so k
right-hand sides are split into contiguous groups of whole blocks, one group per rank, with no collective
on the data path; only the job time is reduced (max over ranks). The global and classical subalgebras
couple all columns and are not sharded this way.
"""
from __future__ import annotations


def shard_columns(k: int, p: int, world: int, rank: int) -> tuple[int, int]:
    """Column range [c0, c1) of `rank`: whole blocks of p columns, as even as possible (leading ranks get one
    block more). Ranks beyond the number of blocks get an empty range."""
    if p < 1 or k % p:
        raise ValueError(f"p={p} must divide k={k}")
    q = k // p
    base, extra = divmod(q, world)
    b0 = rank * base + min(rank, extra)
    nb = base + (1 if rank < extra else 0)
    return b0 * p, (b0 + nb) * p


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's own right-hand sides in the weak-scaling benchmark."""
    return seed + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Job time: the slowest rank's value (a single scalar all-reduce; identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
