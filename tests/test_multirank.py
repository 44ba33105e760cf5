"""The bench's multi-rank path on CPU: world size 2 over gloo (127.0.0.1).  Every rank runs an
independent replica (no data-path collective); the whole-job number takes the slowest rank's
time and the units of all ranks, and under torchrun only rank 0 reports.  No GPU is used.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        ms = bench.max_over_ranks(10.0 * (rank + 1), w, "cpu")       # rank 1 is the slow one
        units = bench.sum_over_ranks(1000.0 + rank, w, "cpu")
        rate = bench.whole_job_rate(units, ms)
        out.put((rank, r, w, lr, ms, units, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, lr, ms, units, rate in res:
        assert (r, w, lr) == (rank, world, rank)
        assert ms == 20.0                        # the slowest rank's time, on every rank
        assert units == 2001.0                   # the units of both ranks
        assert abs(rate - 2001.0 / 0.020) < 1e-6


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.sum_over_ranks(7.0, 1, "cpu") == 7.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    monkeypatch.setattr(bench, "build_workload", lambda a: (_ for _ in ()).throw(AssertionError("did work")))
    bench.main()
    assert capsys.readouterr().out == ""
