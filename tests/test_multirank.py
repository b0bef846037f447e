"""The multi-rank bookkeeping of bench.py on CPU ranks (gloo, world size 2): the
whole-job value takes every rank's points over the slowest rank's time, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, total = bench.aggregate_value(local_ms[rank], steps=10, npoints=1000, world=world)
        out[rank] = (value, total)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_aggregate_value_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    local_ms = [10.0, 15.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, local_ms, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    expect = 2 * 10 * 1000 / (15.0 * 1e-3) / 1e9
    for r in range(2):
        value, total = out[r]
        assert total == 15.0
        assert abs(value - expect) <= 1e-12 * expect


def test_aggregate_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, total = bench.aggregate_value(20.0, steps=5, npoints=4_000_000, world=1)
    assert total == 20.0
    assert abs(value - 5 * 4_000_000 / 0.02 / 1e9) < 1e-9


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.parse_args(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
