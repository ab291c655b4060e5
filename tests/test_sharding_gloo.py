"""Multi-rank path on CPU: two gloo ranks split a batch into contiguous
blocks and sum their knot-value gradients; the result equals the gradient
of the whole batch.  Per-rank gradients come from the oracle (no GPU here),
so this checks the splitting and the exchange, not the kernel."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2009_06635_gb300.sharding import allreduce_knot_gradient, shard_bounds


def test_shard_bounds_cover_the_batch():
    for n in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_bounds(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2009_06635_gb300 import synthetic as S

    g = S.grid_full()
    og = oracle.OracleGrid(g)
    x, q2, cot = S.adjoint_inputs(600, g.nflav, 5, 6)
    a, b = shard_bounds(len(x), rank, world)
    local = torch.from_numpy(og.knot_grad(x[a:b], q2[a:b], cot[a:b]))
    allreduce_knot_gradient(local)
    if rank == 0:
        full, gabs = og.knot_grad(x, q2, cot, with_abs=True)
        ok = bool(np.all(np.abs(local.numpy() - full) <= 1e-12 * gabs + 1e-300))
        q.put(ok)
    dist.destroy_process_group()


def test_two_rank_knot_gradient_allreduce():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert q.get() is True
