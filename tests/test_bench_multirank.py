"""The multi-GPU path of bench.py (independent replicas, the slowest rank's
time, whole-job throughput) checked with two gloo ranks on CPU."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (10 + r) ms of build and (2 + 3r) ms of queries
        tb, tq, ts = bench.reduce_max([10.0 + rank, 2.0 + 3 * rank, 12.0 + 4 * rank], dist, "cpu")
        value, qps = bench.whole_job_rates(entries=1000, queries=500, steps=4, world=world,
                                           t_build_ms=tb, t_query_ms=tq)
        out[rank] = (tb, tq, ts, value, qps)
        info = bench.dist_info()
        assert info == (rank, 0, world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        tb, tq, ts, value, qps = res[rank]
        assert (tb, tq, ts) == (11.0, 5.0, 16.0)
        assert value == pytest.approx(2 * 4 * 1000 / 0.011)
        assert qps == pytest.approx(2 * 4 * 500 / 0.005)


def test_single_process_needs_no_group():
    import bench

    assert bench.reduce_max([1.0, 2.0], None, "cpu") == [1.0, 2.0]
    assert bench.whole_job_rates(10, 20, 2, 1, 1000.0, 500.0) == (20.0, 80.0)
