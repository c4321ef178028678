"""The bench's multi-GPU path is replicas only (no exchange in the step):
the timing reduction (slowest replica) and the whole-job rate, checked with
two gloo ranks on CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slower replica
        slowest = bench.max_over_ranks(ms, "cpu")
        ws, r, local = bench._dist()
        out[rank] = (slowest, ws, r, local, bench.whole_job_rate(ws, 4, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for rank in (0, 1):
        slowest, ws, r, local, rate = out[rank]
        assert slowest == 15.0 and ws == 2 and r == rank and local == rank
        assert rate == pytest.approx(2 * 4 * 1e3 / 15.0)


def test_single_process_passthrough():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_rate(1, 4, 10.0) == pytest.approx(400.0)
