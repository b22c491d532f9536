"""The N > 1 path of bench.py is independent replicas: every rank times its
own copy of the workload and the job reports all ranks' work over the slowest
rank's time.  Two gloo ranks on the CPU check that aggregation."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank], dist, "cpu")
        rate = bench.job_rate(world, 1000.0, slowest)
        q.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_slowest_time_and_whole_job_rate():
    world, times = 2, [1.5, 2.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in out:
        assert slowest == pytest.approx(2.0)
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_one_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(1, 10.0, 2.0) == 5.0
