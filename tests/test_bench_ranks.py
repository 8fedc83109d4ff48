"""The multi-rank side of bench.py on CPU ranks (gloo, world size 2): under torchrun every rank runs an
independent model instance (replicas only, no collective on the data path), the job's rate is the units of all
ranks over the slowest rank's time, and the reference arm runs on rank 0 alone."""
import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import argparse

    import bench
    g = bench.RankGroup(dist, "cpu")
    g.barrier()
    mx = g.max(1.5 + rank)                                   # 1.5 on rank 0, 2.5 on rank 1
    seconds = 2.0 if rank == 0 else 4.0                     # rank 1 is the slow one
    rate = bench.whole_job_rate(100.0, seconds, g)          # 2 ranks x 100 units / 4 s
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        if rank != 0:   # the reference arm: every rank but 0 returns at once, without work or output
            bench.run_reference(argparse.Namespace(steps=1, warmup=0, gpus=world), rank, world)
    results[rank] = (g.world, g.rank, mx, rate, out.getvalue())
    dist.destroy_process_group()


def test_two_cpu_ranks():
    world = 2
    with mp.Manager() as man:
        results = man.dict()
        mp.spawn(_worker, args=(world, _free_port(), results), nprocs=world, join=True)
        res = dict(results)
    for r in range(world):
        w, rk, mx, rate, out = res[r]
        assert (w, rk) == (world, r)
        assert mx == 2.5
        assert rate == pytest.approx(50.0)
        assert out == ""


def test_single_process_group():
    sys.path.insert(0, ROOT)
    import bench
    g = bench.RankGroup()
    g.barrier()
    assert (g.world, g.rank) == (1, 0)
    assert g.max(3.25) == 3.25
    assert bench.whole_job_rate(10.0, 2.0, g) == 5.0
