"""Data parallelism over query points (one process per GPU).

Query points and pixels are independent.  Rank r of R takes the contiguous
range ``shard_range(N, r, R)`` and bakes it with ``point_base = lo``: the
Philox counters carry global point indices, so every shading value equals
the single-process one and the bake has no exchange on its data path.

Two results are sums over all pixels and need one exchange each when the
pixels are sharded: the render loss (Eq. 14, a sum over points and
channels) and the per-triangle error (Sec. 4.4, sums of squared errors and
pixel counts per triangle).  The gradients with respect to per-pixel
material parameters need none: each rank's pixels own their parameters.
"""
from __future__ import annotations

import torch


def shard_range(N: int, rank: int, world: int):
    """[lo, hi) of rank's contiguous share of N items (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank %d of %d" % (rank, world))
    base, extra = divmod(int(N), world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _all_reduce_sum_(t: torch.Tensor, group=None) -> torch.Tensor:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def global_loss(loss: torch.Tensor, group=None) -> torch.Tensor:
    """Sums the ranks' partial losses (float64 [1]) in place; every rank gets the total."""
    return _all_reduce_sum_(loss, group)


def global_tri_error(err: torch.Tensor, count: torch.Tensor, group=None):
    """Sums the ranks' per-triangle error sums (float64 [T]) and pixel counts
    (int32 [T]) in place; every rank gets the totals."""
    _all_reduce_sum_(err, group)
    _all_reduce_sum_(count, group)
    return err, count
