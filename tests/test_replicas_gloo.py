"""The multi-process path of the benchmark on CPU (gloo, world size 2): the
path shards into independent replicas (no collective on the data path), so
what the ranks share is the barrier around the timed region, the max of the
step time over ranks and the whole-job aggregate."""
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
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)   # rank 1 is the slow replica
        value = bench.whole_job_tflops(2.0e12, world, ms)      # 2 TFLOP per rank per step
        bench.barrier(world)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_work():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == pytest.approx(15.0)
        # 2 ranks x 2 TFLOP in 15 ms
        assert value == pytest.approx(2 * 2.0 / 15e-3)


def test_single_process_needs_no_process_group():
    import bench
    bench.barrier(1)
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_tflops(1e12, 1, 1000.0) == pytest.approx(1.0)
