"""The benchmark's multi-rank reduction on CPU (gloo, world size 2).

A mesh does not shard, so N ranks run N independent replicas; the whole-job
value is N x faces / (slowest rank's time).  No GPU involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [40.0, 55.0][rank]                       # rank 1 is the slow one
        got = bench.max_over_ranks(ms, device="cpu")
        out[rank] = (got, bench.weak_value(1_310_720, world, got / 1))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_weak_value():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        ms, v = out[r]
        assert ms == 55.0
        assert v == pytest.approx(2 * 1_310_720 / 0.055 / 1e6)


def test_single_process_identity():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.weak_value(1e6, 1, 1000.0) == pytest.approx(1.0)
