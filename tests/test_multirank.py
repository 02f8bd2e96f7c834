"""The N > 1 path of bench.py (replicas: every rank runs the same workload, the job's time is
the slowest rank's) with two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench._barrier_world() == world          # the sub-workloads' barrier and world size
    ms_local = 10.0 + 5.0 * rank                     # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local)
    value = bench.job_throughput(1000, ms, world)
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 15.0                             # max over ranks
        assert value == pytest.approx(2 * 1000 / 15e-3)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench._barrier_world() == 1
    assert bench.job_throughput(300, 1.5, 1) == pytest.approx(2e5)
