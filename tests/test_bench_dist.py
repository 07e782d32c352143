"""The bench's multi-rank logic on the host: two gloo ranks on 127.0.0.1.

Each rank reports its own units and time; the whole-job value is the sum of the
units over the slowest rank's time, and the reference arm runs on rank 0 only.
"""
import contextlib
import io
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    world, r, _ = bench.dist_init("gloo")
    bench.barrier(world)
    # rank 0: 1000 units in 2 s, rank 1: 3000 units in 5 s
    value, tot, mx = bench.whole_job(1000 * (2 * rank + 1), 2.0 + 3.0 * rank, world)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        if rank != 0:
            bench.run_reference(None, world, rank)    # other ranks leave without work
    q.put((r, value, tot, mx, out.getvalue()))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_whole_job_value():
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tot, mx, printed in res:
        assert tot == 4000.0 and mx == 5.0
        assert value == pytest.approx(800.0)
        assert printed == ""
    assert [r[0] for r in res] == [0, 1]


def test_single_rank_needs_no_process_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    world, rank, local = bench.dist_init()
    assert (world, rank, local) == (1, 0, 0)
    assert bench.whole_job(10, 2.0, 1) == (5.0, 10.0, 2.0)
