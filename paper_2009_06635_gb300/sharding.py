"""Splitting query batches over ranks (one process per GPU).

Query points are independent -- PDFFlow evaluates every (x, Q^2) on its own
(Sec. 2.2) -- so a batch splits into contiguous blocks, one per rank, and the
forward evaluation needs no exchange at all (weak scaling).  The one step of
the path that couples ranks is the adjoint's gradient with respect to the
knot values, a sum over all points of all ranks: each rank accumulates its
block with xfxq2_all_flavours_vjp, then the ranks add their buffers
(allreduce_knot_gradient).
"""
from __future__ import annotations


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of rank's contiguous block; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_knot_gradient(grad_values, group=None):
    """Sum a knot-value gradient buffer over all ranks, in place."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad_values, op=dist.ReduceOp.SUM, group=group)
    return grad_values


def sharded_vjp(grid, x, q2, cot, grad_values, rank: int, world: int, group=None):
    """Adjoint over a batch split across ranks: this rank evaluates its block
    of (x, q2, cot) and all ranks end with the full knot-value gradient.
    Returns this rank's (start, stop, grad_x, grad_q2)."""
    import torch

    from .pdf import xfxq2_all_flavours_vjp

    start, stop = shard_bounds(x.shape[0], rank, world)
    xs, qs, cs = x[start:stop].contiguous(), q2[start:stop].contiguous(), cot[start:stop].contiguous()
    gx, gq = torch.empty_like(xs), torch.empty_like(qs)
    xfxq2_all_flavours_vjp(grid, xs, qs, cs, gx, gq, grad_values)
    allreduce_knot_gradient(grad_values, group)
    return start, stop, gx, gq
