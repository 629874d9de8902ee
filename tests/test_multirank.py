"""The N > 1 path of bench.py on CPU: two gloo ranks take the slowest rank's time and
report the whole-job throughput; under torchrun the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    t_local = 1.0 + rank  # rank 1 is the slower
    t_max = bench.max_over_ranks(t_local, torch.device("cpu"))
    value = bench.whole_job_value(1000, 10, ws, t_max)
    out[rank] = (ws, r, t_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(worker, args=(2, free_port(), out), nprocs=2, start_method="spawn")
    assert out[0][0] == 2 and out[1][1] == 1
    assert out[0][2] == out[1][2] == 2.0
    assert out[0][3] == out[1][3] == 1000 * 10 * 2 / 2.0


def test_single_process_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_value(10, 2, 1, 4.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(workload="kpp", steps=1, warmup=0)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
