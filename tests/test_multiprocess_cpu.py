"""The replicated multi-GPU path of bench.py (one process per GPU, weak scaling,
no data-path collective) on CPU: two gloo ranks check that every rank gets the
slowest rank's time and that the job's throughput counts the units of all
ranks.  No GPU is used."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank          # the second rank is slower
        job_ms = bench.max_over_ranks(local_ms, dist, "cpu")
        dist.barrier()
        results[rank] = (job_ms, bench.job_throughput(1000.0, world, job_ms))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    results = manager.dict()
    mp.start_processes(_rank_main, args=(world, port, results), nprocs=world, start_method="spawn", join=True)
    assert len(results) == world
    for rank in range(world):
        job_ms, thr = results[rank]
        assert job_ms == 15.0                  # max over ranks, on every rank
        assert thr == pytest.approx(2 * 1000.0 / 0.015)  # units of both ranks / job time


def test_single_rank_throughput():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(997002999, 1, 171.3) == pytest.approx(997002999 / 0.1713)
