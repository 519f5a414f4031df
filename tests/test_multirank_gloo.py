"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2).

On several GPUs every rank inpaints its own image (replicas, weak scaling);
the only cross-rank operations are a barrier and the max-over-ranks
reduction of the timed region. Both are exercised here without a GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
        mine = bench.shard(256, rank, world)
        q.put((rank, slowest, mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_is_the_max_and_shards_partition_the_batch():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [15.0, 15.0]
    a, b = res[0][2], res[1][2]
    assert not set(a) & set(b)
    assert sorted(a + b) == list(range(256))
    assert abs(len(a) - len(b)) <= 1


def test_single_rank_helpers_without_a_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("n,world", [(256, 3), (7, 4), (0, 2)])
def test_shards_cover_every_image_once(n, world):
    import bench
    got = sorted(i for r in range(world) for i in bench.shard(n, r, world))
    assert got == list(range(n))
