"""The benchmark's multi-rank logic on the CPU with two gloo ranks: the path
does not shard (replicas only), so a run on N GPUs reports the slowest rank's
time, and the reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench._max_over_ranks(values[rank], world, "cpu")
    finally:
        dist.destroy_process_group()


def test_slowest_rank_time_over_two_gloo_ranks():
    port = _free_port()
    values = [0.75, 1.25]
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(2, port, values, out), nprocs=2, join=True)
        assert dict(out) == {0: 1.25, 1: 1.25}


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench._max_over_ranks(0.5, 1, "cpu") == 0.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.reference_arm(bench._args()) == 0
    assert capsys.readouterr().out == ""
