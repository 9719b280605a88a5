"""The multi-rank benchmark path on CPU: two gloo ranks (replicas of the
workload) agree on the slowest rank's time and on the whole-job throughput."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, "cpu")
    v = bench.aggregate_value(10, world, ms)
    q.put((rank, ms, v))
    dist.destroy_process_group()


def test_two_rank_max_time_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    # 10 units per rank x 2 ranks over 0.15 s
    assert all(abs(o[2] - 20 / 0.15) < 1e-9 for o in out)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.aggregate_value(5, 1, 1000.0) == 5.0
