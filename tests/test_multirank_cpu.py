"""The N > 1 bench path on CPU: two gloo ranks (one process each, 127.0.0.1)
aggregate a timed region the way bench.py does under torchrun -- the slowest
rank's time, every rank's pairs -- and the reference arm runs on rank 0 only."""
import os
import socket

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
    import sys

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, pairs = 10.0 + 5.0 * rank, 1000.0 * (rank + 1)
        ms_job, pairs_job = bench.job_totals(dist, ms, pairs, "cpu")
        e2e = bench.slowest(dist, 0.5 + rank, "cpu")
        out[rank] = (ms_job, pairs_job, e2e)
        # the reference arm: ranks other than 0 return at once without work
        if rank != 0:
            class A:
                warmup, steps, gpus = 3, 1, world
            bench.run_reference(A, rank, world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms_job, pairs_job, e2e = out[r]
        assert ms_job == 15.0 and pairs_job == 3000.0 and e2e == 1.5


def test_one_process_totals_pass_through():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_totals(None, 7.0, 11.0, "cpu") == (7.0, 11.0)
    assert bench.slowest(None, 2.5, "cpu") == 2.5
