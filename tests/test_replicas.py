"""The replicas-only multi-GPU form of bench.py: each rank solves its own
pair, and the job's time is the slowest rank's.  The aggregation runs here
on CPU with two gloo ranks (no GPU)."""
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


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench.dist_env()
        seconds = 1.0 + rank          # rank 1 is the slow replica
        t = bench.max_over_ranks(seconds, got_ws, device="cpu")
        out[rank] = (got_ws, got_rank, t, bench.job_rate(10, got_ws, t))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True,
                       start_method="spawn")
    for rank in range(ws):
        got_ws, got_rank, t, rate = out[rank]
        assert (got_ws, got_rank) == (ws, rank)
        assert t == 2.0                    # the slowest rank's time on every rank
        assert rate == ws * 10 / 2.0       # whole-job units / job time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(7, 1, 2.0) == 3.5
