"""The multi-GPU form of bench.py (replicas, one process per GPU) on CPU: two gloo ranks reduce
their timed regions with MAX and report the whole job's cell-steps; the reference arm does
its work on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.job_time_ms(times[rank], world, device="cpu")
    out[rank] = (t, bench.job_value(world, 1000, 4, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    times = [120.0, 150.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        got = dict(out)
    for rank in range(world):
        t, v = got[rank]
        assert t == 150.0
        assert v == pytest.approx(world * 1000 * 4 / 0.150)


def test_single_rank_keeps_its_time():
    assert bench.job_time_ms(42.0, 1) == 42.0
    assert bench.job_value(1, 10, 2, 1000.0) == pytest.approx(20.0)


def test_reference_arm_works_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None) == 0  # returns before touching the oracle
