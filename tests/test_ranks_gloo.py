"""The host side of multi-process runs, on CPU with two gloo ranks: the timed
region's time is the maximum over ranks on every rank, and the batched
sweep's shards partition the instance list with no instance on two ranks
(no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.ranks_max(dist, 10.0 + 5.0 * rank, "cpu")
    shards = [None] * world
    dist.all_gather_object(shards, bench.shard(512, rank, world))
    q.put((rank, m, shards))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_shards(world):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    env_path = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = env_path + (os.pathsep + old if old else "")
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    try:
        for p in procs:
            p.start()
    finally:
        if old:
            os.environ["PYTHONPATH"] = old
        else:
            del os.environ["PYTHONPATH"]
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, shards in got:
        assert m == 10.0 + 5.0 * (world - 1)          # every rank sees the slowest rank's time
        flat = sorted(i for sh in shards for i in sh)
        assert flat == list(range(512))                 # a partition: every instance once
        assert all(len(sh) == 512 // world for sh in shards)


def test_single_process_helpers():
    import bench
    assert bench.ranks_max(None, 3.5) == 3.5
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.shard(5, 1, 2) == [1, 3]
