"""Multi-rank paths on CPU: two gloo ranks split a batch into contiguous
blocks and sum their knot-value gradients (the result equals the gradient of
the whole batch), and split a Monte Carlo run into event ranges and sum their
weight sums (the result equals one run over all events).  Per-rank values
come from the oracles (no GPU here), so this checks the splitting and the
exchange, not the kernels."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2009_06635_gb300.sharding import allreduce_knot_gradient, allreduce_mc_sums, mc_event_range, shard_bounds


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


def _mc_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from oracle import mc
    from paper_2009_06635_gb300 import synthetic as S

    g = S.grid_full()
    og = oracle.OracleGrid(g)
    cfg = (13000.0, 1e-6, 100.0, 2024)
    per = 3000
    first, count = mc_event_range(rank, per)
    w = mc.weights(og, g.pids, *cfg, first, count, g.x_knots[-1])
    tot = allreduce_mc_sums(mc.sums(w))
    if rank == 0:
        whole = mc.sums(mc.weights(og, g.pids, *cfg, 0, world * per, g.x_knots[-1]))
        ok = all(abs(a - b) <= 1e-12 * whole[2] for a, b in zip(tot[:1] + tot[2:], whole[:1] + whole[2:]))
        ok = ok and abs(tot[1] - whole[1]) <= 1e-12 * whole[1]
        q.put(ok)
    dist.destroy_process_group()


def test_two_rank_mc_sums_allreduce():
    assert mc_event_range(3, 10) == (30, 10)
    assert allreduce_mc_sums([1.0, 2.0, 3.0]) == [1.0, 2.0, 3.0]  # no process group: unchanged
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_mc_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get() is True

