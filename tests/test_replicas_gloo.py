"""The multi-GPU path is replicas only: every rank solves the same workload
and bench.py reports the whole job as the units of all ranks over the
slowest rank's time.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) x 10 ms per step
        ms = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
        q.put((rank, ms, bench.whole_job_rate(world * 4, ms / 1000.0)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time():
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
    assert [o[1] for o in out] == [20.0, 20.0]
    # 2 ranks x 4 RHS in 20 ms: 400 RHS/s for the whole job
    assert all(o[2] == pytest.approx(400.0) for o in out)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(10, 0.5) == 20.0
