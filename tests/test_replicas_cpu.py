"""The N > 1 path of bench.py (replicas only: every rank runs the same step on
its own GPU) on CPU with gloo, world size 2: the job time is the slowest
rank's, and the whole-job throughput counts every rank's work once."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is slower
    t = bench.max_over_ranks(local_ms, "cpu")
    q.put((rank, t, bench.whole_job_tflops(2.0e12, world, t)))
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value in out:
        assert t == 150.0
        assert value == pytest.approx(2.0e12 * 2 / 0.150 / 1e12)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, "cpu") == 12.5
    assert bench.whole_job_tflops(1e12, 1, 1000.0) == pytest.approx(1.0)
