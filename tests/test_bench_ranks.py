"""bench.py's multi-rank host logic on CPU: two gloo ranks (no GPU).

With N ranks every rank sweeps its own replica (weak scaling, no data-path
collective); the job's time is the slowest rank's, and the value is ns per
flip over the flips of all ranks.  The reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.combine_ranks(local_ms[rank], steps=5, n_sites=16, world=world, dist=dist)
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_count_all_flips():
    world = 2
    local_ms = [10.0, 20.0]
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, free_port(), local_ms, out), nprocs=world, join=True)
    for rank in range(world):
        total, per_step, value = out[rank]
        assert total == 20.0
        assert per_step == 4.0
        assert value == pytest.approx(20.0 * 1e6 / (5 * world * 16))


def test_single_rank_needs_no_collective():
    assert bench.combine_ranks(7.0, steps=7, n_sites=4, world=1) == (7.0, 1.0, 7.0 * 1e6 / (7 * 4))


def test_dist_setup_reads_the_launcher_environment(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_setup() == (4, 3, 1)


def test_reference_arm_does_no_work_off_rank_zero(capsys):
    class Args:
        steps, warmup = 1, 3
    bench.run_reference(Args, world=2, rank=1)
    assert capsys.readouterr().out == ""
