"""bench.py's multi-rank aggregation on CPU: two gloo ranks (replicas, as under
torchrun) agree on the slowest rank's time, and the job's throughput counts
every rank's units over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench

        ms = bench.max_over_ranks(times[rank], ws, device="cpu")
        bench.barrier(ws)
        out[rank] = (ms, bench.job_throughput(1000, ms, ws))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ws = 2
    times = [3.0, 5.0]
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, port, times, out), nprocs=ws, join=True,
                       start_method="spawn")
    for r in range(ws):
        ms, value = out[r]
        assert ms == 5.0  # the slowest rank
        assert value == pytest.approx(2 * 1000 / 5e-3)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_throughput(100, 2.0, 1) == pytest.approx(5e4)
