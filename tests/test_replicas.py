"""The multi-GPU mode of the benchmark is replicas (independent solvers, one per GPU; the
solve of one system does not shard).  Its host-side aggregation -- the slowest rank's timed
region, every rank's solves -- is exercised here with two gloo ranks on the CPU; the
reference arm does its work on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 1000.0 + 250.0 * rank          # rank 1 is the slower replica
    total, rate = bench.replica_rate(local_ms, 10, "cpu")
    out[rank] = (total, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        total, rate = out[r]
        assert total == 1250.0                 # the slowest rank's timed region
        assert rate == pytest.approx(world * 10 / 1.25)


def test_replica_rate_single_process():
    import bench
    total, rate = bench.replica_rate(500.0, 5)
    assert total == 500.0 and rate == pytest.approx(10.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"workload": "sphere_small", "steps": 1, "warmup": 0})()
    bench.run_reference(args)                  # returns at once on a non-zero rank
    assert capsys.readouterr().out == ""
