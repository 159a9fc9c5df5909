"""The multi-GPU path is replicas only: host logic checked with two gloo ranks on
the CPU (sharding of independent views, the max-over-ranks timing reduction)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2405_05446_gb300 import replicas as R


def test_shard_covers_every_view_once():
    for n in (0, 1, 7, 8, 33):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in R.shard(n, r, world))
            assert got == list(range(n))
            sizes = [len(R.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        R.shard(4, 2, 2)


def test_aggregate_without_process_group():
    out = R.aggregate(10.0, 2.0)
    assert out["value"] == 5.0 and out["world"] == 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        views = R.shard(10, rank, world)
        seconds = [1.5, 2.5][rank]
        out = R.aggregate(float(len(views)), seconds)
        q.put((rank, views, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_all_views_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, v0, o0), (r1, v1, o1) = res
    assert sorted(v0 + v1) == list(range(10)) and not set(v0) & set(v1)
    for o in (o0, o1):
        assert o["world"] == 2 and o["units"] == 10.0 and o["seconds"] == 2.5
        assert abs(o["value"] - 4.0) < 1e-12
