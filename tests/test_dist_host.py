"""Host logic of the multi-process benchmark on CPU: world_size 2 over gloo (no GPU).  Each rank
trains its own replica (replicas only); the job's time is the slowest rank's and its throughput
counts every rank's points."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench._env_rank()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, w, torch.device("cpu"))
        dist.barrier()
        q.put((rank, r, w, lr, ms, bench.job_throughput(1 << 18, 4, w, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_points():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r_, r, w, lr, ms, value) in enumerate(out):
        assert (r, w, lr) == (rank, 2, rank)
        assert ms == 15.0                                   # max over the ranks' 10 and 15 ms
        assert value == pytest.approx((1 << 18) * 4 * 2 / 15e-3)


def test_single_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5
    assert bench.job_throughput(1000, 10, 1, 2.0) == pytest.approx(5e6)
