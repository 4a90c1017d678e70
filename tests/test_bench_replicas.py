"""Multi-rank logic of bench.py on CPU: replicas aggregated over a gloo group
(world size 2), and the reference arm's rank handling."""

import os
import socket
import sys
import types

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


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 10 (r + 1) ms for its 1e9 units
    val, ms = bench.replica_value(10.0 * (rank + 1), 1e9, world, dist, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{val} {ms}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_replica_value_max_over_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        val, ms = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert ms == pytest.approx(20.0)                       # slowest rank
        assert val == pytest.approx(2 * 1e9 / 20e-3 / 1e9)    # units of all ranks / job time


def test_replica_value_single_rank():
    val, ms = bench.replica_value(4.0, 2e9, 1)
    assert ms == 4.0 and val == pytest.approx(2e9 / 4e-3 / 1e9)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    a = types.SimpleNamespace(order=4, gpus=2, steps=1, warmup=1)
    assert bench.run_reference(a) == 0
    assert capsys.readouterr().out == ""


def test_oracle_processes_time_concurrent_copies():
    """The CPU baseline's timing helper: independent spawned oracle processes
    (one thread each) on a tiny sample, aggregated over the slowest one."""
    val, t_rhs, used = bench.oracle_processes(2, 1, 2, 0, 1)
    assert used == 2 and t_rhs > 0
    dof = 2 ** 3 * 2 ** 3 * 5
    assert val == pytest.approx(2 * dof / t_rhs / 1e9, rel=1e-9)
