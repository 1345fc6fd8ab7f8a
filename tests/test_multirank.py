"""The benchmark's multi-process path (one process per GPU, independent
replicas) on the CPU: two gloo ranks combine their figures the way the
GPU ranks do over NCCL -- the slowest rank's times, every rank's work -- and
the reference arm runs on rank 0 only."""
from __future__ import annotations

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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: times (10 + r, 5 + 2 r) ms, 1000 (r + 1) entries, 7 + r launches
    res = bench.combine_ranks(10.0 + rank, 5.0 + 2 * rank, 1000.0 * (rank + 1), 7 + rank, world,
                              torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = res


def test_two_gloo_ranks_combine_like_the_gpu_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        total, static, edges, launches = res[r]
        assert total == 11.0 and static == 7.0          # the slowest rank
        assert edges == 3000.0 and launches == 15       # all ranks' work


def test_single_process_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(1.0, 2.0, 3.0, 4, 1, None) == (1.0, 2.0, 3.0, 4)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"scale": 10, "steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
