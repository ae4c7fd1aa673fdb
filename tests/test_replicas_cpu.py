"""The multi-process path of bench.py: every rank runs an independent replica
of the solver steps (the method's product does not need data from other
ranks at one GPU per problem), the job's time is the slowest rank's, and the
whole-job rate counts the units of every rank.  Checked with two gloo ranks
on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(local[rank], dist, "cpu")
        out.put((rank, t, bench.job_throughput(1000.0, t, world)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    local = [0.25, 0.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, local, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 0.5
        assert rate == pytest.approx(2 * 1000.0 / 0.5)


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.3) == 0.3
    assert bench.job_throughput(10.0, 2.0, 1) == 5.0
