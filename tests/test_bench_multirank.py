"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own independent problems.
The job time is the slowest rank's, and the whole-job rate counts every rank's units."""
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


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    w, r, loc = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        ms = 100.0 + 50.0 * rank                    # rank 1 is the slower one
        job_ms = bench.max_over_ranks(ms, dist, torch)
        units = bench.sum_over_ranks(10 * (rank + 1), dist, torch)
        rate = bench.whole_job_rate(w, 4, 20, job_ms)
        q.put((r, w, loc, job_ms, units, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_count_every_rank():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(ws))
    for r, (rank, w, loc, job_ms, units, rate) in enumerate(out):
        assert (rank, w, loc) == (r, 2, r)
        assert job_ms == 150.0                       # max over ranks, seen by every rank
        assert units == 30.0                         # 10 + 20
        assert rate == pytest.approx(2 * 4 * 20 / 0.150)


def test_single_process_needs_no_process_group():
    assert bench.max_over_ranks(12.5, None, torch) == 12.5
    assert bench.sum_over_ranks(7.0, None, torch) == 7.0
    assert bench.whole_job_rate(1, 1, 10, 1000.0) == 10.0
