"""The benchmark's multi-GPU aggregation on two CPU ranks (gloo).

bench.py runs one replica per GPU (the path does not shard; see the design notes) and reports
the whole-job throughput: all ranks' bytes divided by the slowest rank's time.  Here two gloo
ranks with different times check that every rank sees the maximum and that the throughput
counts both ranks' work.
"""
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


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank * 0.5, dist, "cpu")
    v = bench.job_throughput(world, 2e9, 10, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_rank_max_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == pytest.approx(1.5)
        assert v == pytest.approx(2 * 2e9 * 10 / 1.5 / 1e9)
