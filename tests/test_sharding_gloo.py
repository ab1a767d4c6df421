"""Multi-process path of the benchmark on CPU (gloo, world size 2): the rank
logic bench.py runs (frequency plan, steps, max-over-ranks timing, gather of
the per-frequency results on rank 0), its own start of N ranks, and failure
detection on the host: a rank that leaves between steps or never joins ends
the others' next collective or rendezvous with an error, not a hang."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

from paper_2412_14973_gb300.sharding import batches, frequency_plan, gather_results, max_over_ranks, shard


def test_shards_partition_and_balance():
    for n, w in [(64, 1), (64, 2), (64, 8), (7, 3), (2, 4)]:
        parts = [shard(n, r, w) for r in range(w)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(n))
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_weak_scaling_plan_gives_every_rank_the_same_rank_mix(world):
    import bench
    wl = bench.PRECISION_FORM
    ranks = wl.ranks(wl.nfreq * world)
    plans = [frequency_plan(wl.nfreq, r, world) for r in range(world)]
    assert sorted(f for p in plans for f in p) == list(range(wl.nfreq * world))
    assert all(len(p) == wl.nfreq for p in plans)
    means = [sum(ranks[f] for f in p) / len(p) for p in plans]
    assert max(means) - min(means) <= 1.0       # same work per GPU (weak scaling)
    for p in plans:
        steps = batches(p, wl.batch)
        assert sorted(f for s in steps for f in s) == sorted(p)
        assert all(len(s) == wl.batch for s in steps)
        # every step spans the rank range: its lowest and highest ranks are
        # within one step's stride of the plan's extremes
        lo, hi = min(ranks[f] for f in p), max(ranks[f] for f in p)
        for s in steps:
            ks = [ranks[f] for f in s]
            assert min(ks) - lo <= (hi - lo) / wl.batch + 1 and hi - max(ks) <= (hi - lo) / wl.batch + 1


def test_batches_reject_a_ragged_split():
    with pytest.raises(ValueError):
        batches(list(range(10)), 4)


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
    mine = frequency_plan(16, rank, world)
    steps = batches(mine, 4)
    records = [{"freq": f, "rank": 8 + f, "iters": 30, "status": 0, "f_final": 1.0 / (1 + f), "f0": 1.0}
               for s in steps for f in s]
    fake_ms = 100.0 + 10.0 * rank + len(mine)
    dist.barrier()
    gathered = gather_results(records, dist)
    out[rank] = (mine, max_over_ranks(fake_ms, dist), gathered)
    dist.destroy_process_group()


def test_gloo_world_size_two():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out[0][0] + out[1][0]) == list(range(32))
    assert out[0][1] == out[1][1] == 100.0 + 10.0 + 16
    got = out[0][2]
    assert [r["freq"] for r in got] == list(range(32))      # every frequency once, on rank 0's host
    assert out[1][2] is None


def test_gather_without_a_process_group_returns_the_records_sorted():
    recs = [{"freq": 3}, {"freq": 1}]
    assert [r["freq"] for r in gather_results(recs)] == [1, 3]


def test_bench_starts_its_own_ranks(monkeypatch):
    # `bench.py --gpus N` outside torchrun starts N copies of itself with the
    # rank environment and a 127.0.0.1 rendezvous
    import bench
    started = []

    class FakeProc:
        def __init__(self, cmd, env):
            started.append((cmd, env))

        def wait(self):
            return 0

    monkeypatch.setattr(bench.subprocess, "Popen", FakeProc)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--gpus", "3", "--steps", "2"])

    class Args:
        gpus = 3

    assert bench.spawn_ranks(Args) == 0
    assert len(started) == 3
    ports = {e["MASTER_PORT"] for _, e in started}
    assert len(ports) == 1
    for r, (cmd, env) in enumerate(started):
        assert env["RANK"] == str(r) and env["LOCAL_RANK"] == str(r) and env["WORLD_SIZE"] == "3"
        assert env["MASTER_ADDR"] == "127.0.0.1"
        assert cmd[1].endswith("bench.py") and cmd[2:] == ["--gpus", "3", "--steps", "2"]


def _failing_worker(rank, world, port, out):
    # rank 1 leaves between steps (after joining, before the gather); rank 0
    # must learn it from its collective (an error or its short timeout), not hang
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)
    try:
        gather_results([{"freq": 0}], dist)
        out[rank] = "no error"
    except Exception as e:  # a lost peer surfaces as a backend error
        out[rank] = "error: " + type(e).__name__


def test_a_rank_that_leaves_is_detected_by_the_others():
    import time
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, out)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung after its peer left"
    assert procs[1].exitcode == 3
    assert out.get(0, "").startswith("error"), out.get(0)
    assert time.time() - t0 < 120


def _lonely_worker(port, out):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=0, world_size=2, timeout=datetime.timedelta(seconds=5))
        gather_results([{"freq": 0}], dist)
        out[0] = "no error"
    except Exception as e:  # the peer never joined: the rendezvous times out
        out[0] = "error: " + type(e).__name__


def test_a_rank_that_never_joins_ends_the_rendezvous_with_an_error():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    p = ctx.Process(target=_lonely_worker, args=(_free_port(), out))
    p.start()
    p.join(120)
    if p.is_alive():
        p.kill()
        pytest.fail("the lone rank hung")
    assert out.get(0, "").startswith("error"), out.get(0)
