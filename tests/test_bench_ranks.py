"""Whole-job aggregation of bench.py under several ranks, on CPU with the gloo backend.

bench.py runs one replica of the workload per GPU (no data-path collective); the only
cross-rank step is the max of the per-rank step times, from which the whole-job throughput is
computed. Here two gloo ranks report different times and must agree on the max and the value.
"""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [2.0, 3.5][rank]
        ms_max = bench.max_over_ranks(ms, torch.device("cpu"))
        out.put((rank, ms_max, bench.job_value(1_000_000, world, ms_max), bench.rank_seed(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [3.5, 3.5]
    assert res[0][2] == res[1][2] == pytest.approx(2 * 1_000_000 / 3.5e-3 / 1e6)
    assert res[0][3] != res[1][3]          # each rank assembles its own mesh


def test_single_process_needs_no_process_group():
    import torch

    import bench

    assert bench.max_over_ranks(1.25, torch.device("cpu")) == 1.25
    assert bench.job_value(8_388_608, 1, 2.0) == pytest.approx(4194.304)
