"""The benchmark's multi-GPU path is replicas (independent measurements, no
data-path collective): two gloo ranks on the CPU check that each rank gets its
own measurement, that the job time is the slowest rank's, and that the
throughput counts every rank's work."""
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
    try:
        local = [10.0 + 5.0 * rank, 20.0 - rank]
        mx = bench.max_over_ranks(local, world)
        seed = bench.rank_workload(rank).seed
        q.put((rank, mx, seed, bench.job_throughput(1e9, world, mx[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, mx0, s0, v0), (r1, mx1, s1, v1) = res
    assert mx0 == mx1 == [15.0, 20.0]
    assert s0 != s1
    assert v0 == v1 == pytest.approx(2e9 / 0.015)
