"""bench.py's multi-rank host logic on CPU with gloo (world size 2): the timed
region is the slowest rank's, the value the whole job's rate, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(times[rank], "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    times = [12.5, 31.0]
    mp.start_processes(_rank_main, args=(world, port, times, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1] == 31.0


def test_job_rate_is_whole_job():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 10 steps x 1e12 flops in 1000 ms -> 20 TFLOP/s
    assert abs(bench.job_rate(1e12, 2, 1000.0, 10) - 20.0) < 1e-12
    assert abs(bench.job_rate(1e12, 1, 1000.0, 10) - 10.0) < 1e-12


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "b": "auto"})()
    assert bench.run_reference(args) == 0
