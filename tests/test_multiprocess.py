"""The N > 1 path of bench.py ("replicas only": every rank advances its own copy of the
workload on its own GPU, no collective on the data path) on CPU with two gloo ranks:
the timing is the slowest rank's on every rank, the whole-job rate counts every rank's
cells, and the reference arm runs on rank 0 only."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 20.0][rank]
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        rate = bench.whole_job_rate(world, 1000, 4, ms)
        # the reference arm: the ranks other than 0 leave at once and print nothing
        out = io.StringIO()
        if rank != 0:
            with redirect_stdout(out):
                rc = bench.run_reference(None)  # returns before it reads its arguments
        else:
            rc = 0
        q.put((rank, ms, rate, rc, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, rc, printed in res:
        assert ms == 20.0  # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 9 * 1000 * 4 / 20e-3)
        assert rc == 0
        if rank != 0:
            assert printed == ""


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
    assert bench.whole_job_rate(1, 10, 2, 1000.0) == pytest.approx(9 * 10 * 2)
