"""Multi-GPU form of the benchmark: replicas only (instances are independent,
no collective on the data path).  The host-side logic is checked with two
gloo ranks on the CPU: timings are reduced with MAX (the job ends with its
slowest rank), the rate counts every rank's units, and the reference arm runs
on rank 0 alone."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]
        mx = bench.max_over_ranks(ms, world, "cpu")
        rate = bench.job_throughput(256 * 10, world, mx)

        class Args:
            steps, warmup, batch, agents = 2, 1, 4, 8
        buf = io.StringIO()
        with redirect_stdout(buf):
            if rank != 0:
                bench.run_reference(Args, rank, world)
        q.put((rank, mx, rate, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_with_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, mx, rate, out = q.get(timeout=120)
        res[rank] = (mx, rate, out)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        mx, rate, out = res[rank]
        assert mx == pytest.approx(20.0)
        assert rate == pytest.approx(2 * 2560 / 0.020)
    assert res[1][2] == ""  # the reference arm prints and runs nothing off rank 0
