"""Replica aggregation of the benchmark on two CPU ranks (gloo): every rank runs an independent copy of the
workload, the job time is the slowest rank's, and the throughput counts all ranks' lattice updates."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        t = bench.replica_max(ms, ws)
        out[rank] = (t, bench.aggregate_glups(1000, 20, ws, t / 1e3))
    finally:
        dist.destroy_process_group()


def test_replica_max_and_aggregate_two_ranks():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        t, v = res[r]
        assert t == 15.0
        assert v == pytest.approx(1000 * 20 * 2 / 0.015 / 1e9)


def test_single_rank_is_identity():
    import bench

    assert bench.replica_max(3.5, 1) == 3.5
    assert bench.aggregate_glups(2_097_152, 200, 1, 0.07) == pytest.approx(2_097_152 * 200 / 0.07 / 1e9)
