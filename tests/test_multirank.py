"""The multi-rank logic of bench.py on CPU (gloo, world size 2): replicas
run independently, the reported time is the slowest rank's and the rate is
the whole job's (weak scaling). The GPU path itself has no data-path
collective; the timing barrier and this max-reduce are its only ones."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 * (rank + 1)            # rank 1 is the slow replica
        dist.barrier()
        ms = bench.max_over_ranks(ms_local, dist, torch.device("cpu"))
        value = bench.whole_job_rate(298248, world, ms)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()   # no fork of this (threaded) process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]                      # every rank reports the same
    ms, value = out[0]
    assert ms == 20.0                            # the slowest rank
    assert value == pytest.approx(2 * 298248 / 0.020)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.whole_job_rate(1000, 1, 500.0) == pytest.approx(2000.0)
