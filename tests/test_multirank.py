"""bench.py's multi-rank plumbing on CPU: two gloo ranks (world size 2).

With N GPUs the bench runs N independent replicas (no data-path collective):
each rank times its own steps, the slowest rank's time is taken (MAX over
ranks), and only rank 0 prints. These tests run that host logic with the gloo
backend on 127.0.0.1.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        assert (w, r, local) == (world, rank, rank)
        # per-rank "times": the slowest rank's value wins on every rank
        m = bench.max_over_ranks(10.0 + 5.0 * rank, world)
        bench.barrier(world)
        # the reference arm: ranks other than 0 return without work or output
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(None)
        out[rank] = (m, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_barrier_and_rank0_only_output():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 0], codes
    assert res[0][0] == 15.0 and res[1][0] == 15.0
    assert res[1][1] == ""


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    bench.barrier(1)
