"""Host logic of bench.py's N > 1 path (independent replicas, one per GPU),
exercised with world_size 2 on the gloo backend on CPU.  The transform itself
has no cross-GPU exchange on one device, so the only multi-rank logic is the
barrier / max-over-ranks timing and rank-0-only reporting."""
import io
import json
import os
import sys
import contextlib

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [10.0 + rank, 20.0 - rank]  # per-rank ms: rank 1 slower in the first value
    got = bench.reduce_over_ranks(mine, world)
    dist.barrier()
    # the reference arm: only rank 0 works and prints
    buf = io.StringIO()

    class A:
        steps, warmup = 1, 0
    with contextlib.redirect_stdout(buf):
        if rank != 0:
            bench.run_reference(A, rank, world)
    q.put((rank, got, buf.getvalue()))
    dist.destroy_process_group()


def test_max_over_ranks_and_rank0_reporting():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, out in res:
        assert got == [11.0, 20.0]  # max over the two ranks, element-wise
        if rank != 0:
            assert out == ""  # non-zero ranks print nothing


def test_job_value_scales_with_replicas():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_value(12.0, 1) == 12.0
    assert bench.job_value(12.0, 4) == 3.0
    assert bench.reduce_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
