"""The benchmark's multi-rank logic on two CPU ranks (gloo): the job's time is the slowest rank's,
the job's rate counts every rank's units, and only rank 0 runs and prints the reference arm."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(10.0 + 5.0 * rank)
        rate = bench.whole_job_rate(1000.0, world, ms)
        out = io.StringIO()
        with redirect_stdout(out):   # the reference arm: ranks other than 0 leave without work
            if rank != 0:
                bench.run_reference(None, None)
        q.put((rank, ms, rate, out.getvalue(), bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, out, env in res:
        assert ms == 15.0                       # the slower rank's time, on every rank
        assert rate == pytest.approx(2 * 1000.0 / 0.015)
        assert env == (rank, 2, rank)
    assert res[1][3] == ""                      # rank 1 printed nothing for the reference arm


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(99.2e6, 1, 56.0) == pytest.approx(99.2e6 / 0.056)
