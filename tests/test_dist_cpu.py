"""The multi-rank bookkeeping of bench.py on CPU ranks (gloo, world size 2).

With more than one GPU every rank runs its own independent replica grid; the
job's throughput is all ranks' moves divided by the slowest rank's time.
This runs that reduction across two CPU processes.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    local_moves = [1_000_000, 3_000_000][rank]
    value, tmax = bench.job_throughput(local_ms, local_moves, world, "cpu")
    out[rank] = (value, tmax)
    dist.destroy_process_group()


def test_job_throughput_two_ranks():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        value, tmax = out[r]
        assert tmax == 250.0
        assert value == pytest.approx(4_000_000 / 0.25)


def test_single_rank_combination():
    import bench
    assert bench.combine_rank_results([10.0, 20.0], [5, 5]) == (10 / 0.02, 20.0)
    assert bench.job_throughput(20.0, 10, 1, "cpu") == (10 / 0.02, 20.0)
