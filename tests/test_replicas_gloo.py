"""Multi-rank (replica) path of bench.py on CPU: two gloo ranks report
different step times; every rank must get the slowest rank's time and the
whole-job value N * steps / max_time. The solve itself does not shard (each
GPU runs an independent replica), so this reduction is the only exchange."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, ms, w = bench.aggregate_over_ranks(1000.0 * (rank + 1), 3, dist)
    q.put((rank, value, ms, w))
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms, w in out:
        assert w == 2 and ms == 2000.0
        assert value == pytest.approx(2 * 3 / 2.0)


def test_single_process_aggregation():
    import bench
    value, ms, w = bench.aggregate_over_ranks(500.0, 2, None)
    assert (w, ms) == (1, 500.0) and value == pytest.approx(4.0)


def test_shard_problems_partition_and_balance():
    # C5 sizes: N uniform in [256, 4096], cost N^2 (nev + nex)
    import bench
    Ns = bench.batch_sizes(96)
    costs = [float(N) ** 2 * (-(-N // 20) - (-N // 40)) for N in Ns]
    for world in (1, 2, 3, 4, 8, 97):
        shards = bench.shard_problems(costs, world)
        assert len(shards) == world
        flat = sorted(k for s in shards for k in s)
        assert flat == list(range(96))  # every problem exactly once
        loads = [sum(costs[k] for k in s) for s in shards]
        # list scheduling bound: no rank exceeds the average by more than one problem
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-6 * sum(costs)


def _shard_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    Ns = bench.batch_sizes(96)
    costs = [float(N) ** 2 * (-(-N // 20) - (-N // 40)) for N in Ns]
    mine = bench.shard_problems(costs, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    q.put((rank, gathered))
    dist.destroy_process_group()


def test_two_rank_batch_sharding_is_consistent():
    # every rank derives its shard on its own; together the shards cover all
    # problems once (no collective is needed on the data path)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered in out:
        assert sorted(k for s in gathered for k in s) == list(range(96))
        assert not set(gathered[0]) & set(gathered[1])
