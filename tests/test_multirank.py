"""Multi-rank host logic of bench.py on CPU: two gloo ranks.

The path shards into independent instances (replicas in the step mode, dealt-out
ensemble members in the ensemble mode); the only cross-rank steps are the
max-over-ranks time and the sum of the units, which these tests check.
"""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 10 (r + 1) units in 1 + r seconds
        rate, units, secs = bench.job_rate(10.0 * (rank + 1), 1.0 + rank, dist, "cpu")
        mx = bench.reduce_over_ranks([rank, -rank], "max", dist, "cpu")
        sm = bench.reduce_over_ranks([1.0, rank], "sum", dist, "cpu")
        out[rank] = (rate, units, secs, mx, sm, bench.shard(7, rank, world))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_units_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    units = 10.0 + 20.0
    for r in range(world):
        rate, u, secs, mx, sm, mine = res[r]
        assert u == units
        assert secs == 2.0                 # the slowest rank
        assert rate == pytest.approx(units / 2.0)
        assert mx == [1.0, 0.0]
        assert sm == [2.0, 1.0]
    # the ensemble deal covers every instance exactly once
    dealt = sorted(res[0][5] + res[1][5])
    assert dealt == list(range(7))
    assert set(res[0][5]).isdisjoint(res[1][5])


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(12.0, 3.0) == (4.0, 12.0, 3.0)
    assert bench.reduce_over_ranks([1, 2], "max") == [1.0, 2.0]
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
