"""The multi-GPU path of bench.py is replicas only (one independent solve per rank, no
data-path collective).  Its host logic — the max-over-ranks time of the timed region and
the whole-job throughput — runs here on CPU as two gloo ranks."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(times[rank], dist, "cpu")
    out[rank] = (ms, bench.job_value(world, 1000, 10, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    times = [12.5, 20.0]
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 20.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.020)


def test_single_process_keeps_its_own_time():
    import bench
    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.job_value(1, 100, 4, 2.0) == pytest.approx(100 * 4 / 0.002)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    """Under torchrun only rank 0 of the reference arm times the oracle."""
    import bench

    class A:
        workload = "sod"
        steps = 1
        warmup = 0
        path = "full"

    called = []
    monkeypatch.setattr(bench, "make_workload", lambda name: called.append(name) or None)
    assert bench.run_reference(A(), 1, 2) is None
    assert called == ["sod"]  # the workload is described, the oracle is never built
