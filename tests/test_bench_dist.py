"""The replicated (N>1) benchmark path on CPU: two gloo ranks, the job time is
the slowest rank's and the rate counts every rank's solves."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank            # rank 1 is slower
    m = bench.max_over_ranks(torch, ms, "cpu")
    rate = bench.job_rate(10, world, m)
    out[rank] = (m, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    assert out[0] == out[1]
    assert out[0][0] == pytest.approx(150.0)
    assert out[0][1] == pytest.approx(2 * 10 / 0.150)


def test_single_process_has_no_collective():
    assert bench.max_over_ranks(torch, 12.5, "cpu") == 12.5
    assert bench.job_rate(4, 1, 1000.0) == pytest.approx(4.0)
