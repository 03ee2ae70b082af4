"""The multi-rank path of bench.py (replicas, no collective on the data path) on CPU:
two gloo ranks time different steps; the job time is the slowest rank's and the whole-job
value counts the units of both ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slower replica
        job = bench.max_over_ranks(ms, world, "cpu")
        out[rank] = (job, bench.replica_throughput(1000.0, world, job))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        job, value = res[rank]
        assert job == 15.0
        assert value == pytest.approx(world * 1000.0 / 0.015)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.replica_throughput(10.0, 1, 1000.0) == 10.0


def test_epoch_split_first_and_later():
    import bench
    ms = [10.0, 5.0, 6.0, 12.0, 5.5, 6.5]        # two jobs of three epochs
    first, rest = bench.epoch_split(ms, 3)
    assert first == 11.0 and rest == 5.75
    assert bench.epoch_split([3.0, 4.0], 1) == (3.5, None)
