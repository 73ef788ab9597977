"""The N > 1 bench path runs independent replicas (no collective on the data
path); its host logic (the job's time is the slowest rank's, the job's rate
counts every rank's units, only rank 0 runs the reference arm) is checked here
with two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slower replica
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        rate = bench.job_throughput(24000 * 50, world, ms / 1e3)
        ref_rc = bench.run_reference(None, rank, world) if rank == 1 else 0
        out[rank] = (ms, rate, ref_rc)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_every_rank():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == res[1][1] == pytest.approx(24000 * 50 * 2 / 0.015)
    assert res[1][2] == 0                      # rank 1 of the reference arm exits without work


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(100, 1, 0.5) == 200
