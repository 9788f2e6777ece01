"""The bench's multi-rank accounting on the CPU: two gloo ranks (the replicas
form of `--gpus N`): the step time is the max over ranks and the pixels the
sum; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = bench.reduce_over_ranks(torch, dist, float(rank + 1), "max")
        sm = bench.reduce_over_ranks(torch, dist, float(10 * (rank + 1)), "sum")
        q.put((rank, mx, sm))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_sum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2.0, 30.0), (1, 2.0, 30.0)]


def test_reduce_without_process_group_is_identity():
    sys.path.insert(0, ROOT)
    import torch

    import bench
    assert bench.reduce_over_ranks(torch, None, 3.5, "max") == 3.5


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"gpus": 2, "steps": 1, "warmup": 3})()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
