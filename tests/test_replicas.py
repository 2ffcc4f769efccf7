"""Multi-process replica path of bench.py on the host (gloo, world size 2): replicas process
independent scans with no data-path collective; the whole-job throughput is the units all
ranks processed over the slowest rank's time, and the reference arm runs on rank 0 alone."""
import io
import os
import socket
import sys
from argparse import Namespace
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(Namespace(impl="reference"))
    assert (w, r) == (world, rank)
    assert dist.get_backend() == "gloo"
    # rank r processed 10 * (r + 1) units in (r + 1) seconds
    value, t_max, total = bench.replica_throughput(10.0 * (rank + 1), float(rank + 1), world)
    buf = io.StringIO()
    with redirect_stdout(buf):
        if rank != 0:
            bench.run_reference(Namespace(steps=1, warmup=0, gpus=world, fast=False,
                                          no_graph=False), world, rank)
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, value, t_max, total, buf.getvalue()))


def test_replica_throughput_gloo_world2():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
            pytest.fail("gloo worker did not finish")
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(world))
    for rank, value, t_max, total, printed in out:
        assert t_max == 2.0                 # slowest rank
        assert total == 30.0                # 10 + 20 units
        assert value == 15.0                # whole-job throughput
        if rank != 0:
            assert printed == ""            # the reference arm prints on rank 0 only


def test_replica_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(12.0, 3.0, 1) == (4.0, 3.0, 12.0)
