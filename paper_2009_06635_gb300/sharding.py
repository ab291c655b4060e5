"""Splitting query batches over ranks (one process per GPU).

Query points are independent -- PDFFlow evaluates every (x, Q^2) on its own
(Sec. 2.2) -- so a batch splits into contiguous blocks, one per rank, and the
forward evaluation needs no exchange at all (weak scaling).  The one step of
the path that couples ranks is the adjoint's gradient with respect to the
knot values, a sum over all points of all ranks: each rank accumulates its
block with xfxq2_all_flavours_vjp, then the ranks add their buffers
(allreduce_knot_gradient).  A Monte Carlo integration splits its events the
same way (mc_event_range: disjoint ranges of the counter-based generator)
and adds the three weight sums at the end (allreduce_mc_sums).
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


def mc_event_range(rank: int, events_per_rank: int) -> tuple[int, int]:
    """(first event, count) of a rank: consecutive global event indices, so
    the counter-based generator draws disjoint events on every rank."""
    if rank < 0 or events_per_rank < 0:
        raise ValueError("rank and events_per_rank must be >= 0")
    return rank * events_per_rank, events_per_rank


def allreduce_mc_sums(sums, group=None) -> list:
    """Sum (sum w, sum w^2, sum |w|) over the ranks of the default (or given)
    group; returns the totals as floats (the input unchanged with one rank).
    The sums travel as one FP64 tensor on the backend's device."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return [float(v) for v in sums]
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in sums], dtype=torch.float64, device=dev)
    dist.all_reduce(t, group=group)
    return [float(v) for v in t.cpu()]

