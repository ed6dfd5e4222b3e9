"""The multi-rank path of bench.py on CPU: two gloo ranks run the replicas'
aggregation (barrier, max-over-ranks time, whole-job GB/s) as the GPU ranks
do under torchrun; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    t = bench.max_over_ranks(times[rank], world, torch.device("cpu"))
    out[rank] = (t, bench.whole_job_gbs(2e9, t, world))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, times = 2, [0.5, 0.8]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), times, out), nprocs=world, start_method="spawn")
    for r in range(world):
        t, v = out[r]
        assert t == pytest.approx(0.8)
        assert v == pytest.approx(2e9 * 2 / 0.8e-3 / 1e9)


def test_one_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.25, 1, None) == 1.25
    assert bench.whole_job_gbs(1e9, 1.0, 1) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.main()  # returns without work on a rank other than 0
    assert capsys.readouterr().out == ""
