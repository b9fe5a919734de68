"""The N > 1 path of bench.py runs independent replicas and reports the max over ranks; checked
with two gloo ranks on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        r, w, _ = bench.env_rank()
        out[10 + rank] = r * 100 + w
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.5
    assert out[10] == 2 and out[11] == 102


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25


def _shard_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [float((37 * i) % 101 + 1) for i in range(256)]     # uneven problem sizes
        mine = bench.shard_of(costs, world, rank)
        # every rank's view of every shard (a host-side check only; the data path has no collective)
        views = [None] * world
        dist.all_gather_object(views, [bench.shard_of(costs, world, r) for r in range(world)])
        out[rank] = (mine, views, sum(costs[i] for i in mine))
    finally:
        dist.destroy_process_group()


def test_batch_shards_cover_every_graph_once_on_two_gloo_ranks():
    """The batched configuration splits its independent graphs over the ranks: the shards are
    disjoint, cover all graphs, are computed identically on every rank, and balance the load."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    m0, v0, l0 = out[0]
    m1, v1, l1 = out[1]
    assert v0 == v1 == [[m0, m1], [m0, m1]]
    assert sorted(m0 + m1) == list(range(256))
    assert abs(l0 - l1) <= 101
