"""The multi-process path of bench.py on CPU: two gloo ranks stand in for two
GPUs (replicas of the workload, no data-path collective).  Every rank must
report the slowest rank's time, the whole-job value must count the fluid-node
updates of all ranks, and the reference arm must run on rank 0 alone."""
import argparse
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(times[rank], dist, "cpu")
    q.put((rank, ms, bench.whole_job_mlups(1000, 10, ms, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_the_whole_job_value():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [3.0, 5.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == 5.0
        # 2 ranks x 1000 fluid nodes x 10 steps in 5 ms = 4 MLUPS
        assert value == pytest.approx(4.0)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.whole_job_mlups(1000, 10, 5.0, 1) == pytest.approx(2.0)


def test_reference_arm_prints_nothing_on_other_ranks():
    import bench
    args = argparse.Namespace(workload="throughput", steps=1, warmup=0, gpus=2)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args, rank=1)
    assert buf.getvalue() == ""
