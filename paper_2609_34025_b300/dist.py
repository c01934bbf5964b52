"""Multi-process sharding of tree field integration (one process per GPU).

Channels are independent (tensor fields are integrated coordinatewise), and so
are the trees of a forest, so the work shards with no exchange on the data
path: each rank owns a block of channels (or trees) and runs the whole apply on
its own GPU. The only collectives are the ones a benchmark needs around its
timed region: a barrier and a max-reduce of the elapsed time.
"""
from __future__ import annotations


def channel_block(rank: int, world: int, d: int) -> tuple[int, int]:
    """[c0, c1) of the d channels owned by `rank` (contiguous, sizes differ by at most one)."""
    if not (0 <= rank < world) or d < 0:
        raise ValueError("need 0 <= rank < world and d >= 0")
    base, extra = divmod(d, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def tree_block(rank: int, world: int, n_trees: int) -> tuple[int, int]:
    """[t0, t1) of the trees of a batch owned by `rank`."""
    return channel_block(rank, world, n_trees)


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
