"""The N > 1 bench path on CPU: replicas reduced with gloo (world size 2), no GPU.

The re-ranking path runs as independent replicas (one pipeline per GPU, no data-path
collective); the only cross-rank step is the timing reduction: the job time is the slowest
rank's, and the throughput counts the queries of every replica.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slower replica
    m = bench.max_over_ranks(ms, dist, "cpu")
    v = bench.job_throughput(world, 3368, m)
    dist.barrier()
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_replicas_reduce_max_time_and_sum_queries():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == pytest.approx(15.0)
        assert v == pytest.approx(2 * 3368 / 0.015)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(7.0, None) == 7.0
    assert bench.job_throughput(1, 100, 50.0) == pytest.approx(2000.0)
