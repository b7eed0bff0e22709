"""Host logic of the multi-GPU layout: view shards and the gradient all-reduce, on gloo ranks (CPU)."""
import os
import socket

import numpy as np
import pytest

from paper_2406_12080_b300 import sharding, synth


def _cams(n):
    res = ((1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))
    return [synth.look_camera([0, 0, 0], [0, 0, 1], [0, -1, 0], *res[i % 4], 60.0, 6.0) for i in range(n)]


@pytest.mark.parametrize("n,world", [(32, 1), (32, 2), (32, 8), (7, 2), (3, 4), (0, 2)])
def test_shards_cover_every_view_once_and_balance_pixels(n, world):
    cams = _cams(n)
    seen = []
    loads = []
    for r in range(world):
        lo, part = sharding.shard_views(cams, r, world)
        seen += list(range(lo, lo + len(part)))
        loads.append(sum(c.width * c.height for c in part))
    assert seen == list(range(n))
    if n >= world:
        biggest = max((c.width * c.height for c in cams), default=0)
        assert max(loads) - min(loads) <= 2 * biggest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = {"mean": torch.full((5, 3), float(rank + 1)), "sh": torch.arange(10.0).reshape(2, 5) * (rank + 1),
             "opacity": torch.tensor([rank * 1.0])}
        sharding.allreduce_grads(g)
        q.put((rank, {k: v.numpy().copy() for k, v in g.items()}))
    finally:
        dist.destroy_process_group()


def test_gradient_allreduce_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        np.testing.assert_array_equal(out[r]["mean"], np.full((5, 3), 3.0))
        np.testing.assert_array_equal(out[r]["sh"], np.arange(10.0).reshape(2, 5) * 3)
        np.testing.assert_array_equal(out[r]["opacity"], [1.0])


def _timing_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.rank_barrier(world)
        q.put((rank, bench.rank_max([2.5, 7.0][rank], world, "cpu"), bench.rank_max(rank, 1, "cpu")))
    finally:
        dist.destroy_process_group()


def test_bench_times_the_slowest_rank():
    """The bench's job timings on two gloo ranks: every rank receives the largest of the ranks' times
    (the whole job's), and one rank keeps its own."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_timing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {r: (a, b) for r, a, b in (q.get(timeout=120) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: (7.0, 0.0), 1: (7.0, 1.0)}
