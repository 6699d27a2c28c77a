"""The multi-rank host logic of the benchmark on CPU ranks (gloo, world size 2): each
GPU runs an independent replica (the product has no exchange step), and the whole-job
figures are the slowest rank's time and the summed work of all ranks."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, w = bench.aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1), torch.device("cpu"))
        dist.barrier()
        out.put((rank, t, w))
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 15.0, 300.0), (1, 15.0, 300.0)]


def test_aggregate_single_process_is_identity():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(3.5, 7.0, torch.device("cpu")) == (3.5, 7.0)
