"""Multi-process path of the benchmark on CPU (gloo, world size 2): each rank
takes its own frequencies, the shards cover everything once, and the step time
is the maximum over the ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2412_14973_gb300.sharding import max_over_ranks, shard


def test_shards_partition_and_balance():
    for n, w in [(64, 1), (64, 2), (64, 8), (7, 3), (2, 4)]:
        parts = [shard(n, r, w) for r in range(w)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(n))
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(64, rank, world)
    fake_ms = 100.0 + 10.0 * rank + len(mine)
    dist.barrier()
    out[rank] = (mine, max_over_ranks(fake_ms, dist))
    dist.destroy_process_group()


def test_gloo_world_size_two():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out[0][0] + out[1][0]) == list(range(64))
    assert out[0][1] == out[1][1] == 100.0 + 10.0 + 32
