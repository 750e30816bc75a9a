"""bench.py's multi-rank aggregation with two gloo ranks on CPU: each rank runs
its own replica (no collective on the data path); the job time is the maximum
over ranks and the throughput counts every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = [10.0, 25.0][rank]
    t, value = bench.combine_ranks(local_ms, units_per_rank=1000.0, steps=4)
    dist.barrier()
    out[rank] = (t, value)
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_max_time_and_sums_units():
    ws = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:   # no fork of this threaded process
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        t, value = res[rank]
        assert t == pytest.approx(25.0)
        assert value == pytest.approx(1000.0 * 4 * 2 / 0.025)


def test_single_process_aggregation():
    import bench
    t, value = bench.combine_ranks(20.0, units_per_rank=500.0, steps=10)
    assert t == 20.0 and value == pytest.approx(500.0 * 10 / 0.02)
