"""The N-replica benchmark path on CPU: two gloo ranks (world size 2) agree on
the slowest rank's step time and on the whole-job throughput, and a rank that
raises is reported by the launcher instead of hanging the others."""
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


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow replica
        ms = bench.reduce_max(local_ms, dist, torch.device("cpu"))
        value = bench.whole_job_tflops(world, 2.0e12, ms)
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 15.0
    # 2 ranks x 2 TFLOP per step in 15 ms
    assert out[0][1] == pytest.approx(2 * 2.0 / 0.015)


def _failing_worker(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    if rank == 1:
        raise RuntimeError("replica 1 failed")    # host-side failure, no GPU involved
    dist.destroy_process_group()


def test_a_failing_replica_is_reported():
    with pytest.raises(Exception) as e:
        mp.start_processes(_failing_worker, args=(2, _free_port()), nprocs=2,
                           start_method="spawn", join=True)
    assert "replica 1 failed" in str(e.value) or "process 1" in str(e.value)
