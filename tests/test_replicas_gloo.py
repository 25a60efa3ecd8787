"""Replica runs on several ranks (CPU, gloo, world size 2).

The path does not shard across GPUs here: N ranks run independent replicas
(independent qDRIFT seeds or batches) and only the timing and counts cross
ranks.  This checks that aggregation with real process groups: the job time
is the slowest rank's, the units and launches are summed, and every rank
sees the same numbers; and that the replicas draw different samples.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, units, launches = bench.aggregate_ranks(dist, torch.device("cpu"), 10.0 + 3.0 * rank, 1000 * (rank + 1),
                                                   7 + rank)
        out[rank] = (t, units, launches)
    finally:
        dist.destroy_process_group()


def test_aggregation_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (13.0, 3000, 15)
    # whole-job throughput: all units over the slowest rank's time
    t, units, _ = res[0]
    assert units / (t / 1e3) == pytest.approx(3000 / 0.013)


def test_single_process_aggregation_is_identity():
    assert bench.aggregate_ranks(None, None, 5.0, 10, 3) == (5.0, 10, 3)


def test_replicas_draw_independent_samples():
    # each rank's qDRIFT seed differs, so its rotation stream differs
    w0, w1 = bench.make_workload(0), bench.make_workload(1)
    assert w0[5] != w1[5]
