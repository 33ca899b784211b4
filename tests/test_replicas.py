"""The N > 1 host logic of the benchmark: each rank runs its own replica; the
timing is the maximum over ranks and the throughput the sum of the units all
ranks processed over that time. world_size 2 with gloo on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        bench.barrier(w)
        ms = 100.0 + 50.0 * rank          # this replica's timed milliseconds
        units = 1_000_000 * (rank + 1)    # its cell updates
        out[rank] = (bench.reduce_max(ms, w), bench.reduce_sum(units, w))
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_max_time_and_sum_units():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that may hold threads
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (150.0, 3_000_000.0)
    # the value the benchmark reports: all units over the slowest replica's time
    ms_max, units = res[0]
    assert units / (ms_max / 1e3) == pytest.approx(2.0e7)


def test_single_process_needs_no_process_group():
    assert bench.reduce_max(3.0, 1) == 3.0 and bench.reduce_sum(4.0, 1) == 4.0
