"""The N > 1 path of bench.py on CPU: two gloo ranks, barrier and max-over-ranks timing.

Each rank advances its own replica (no data-path collective); the whole-job throughput is the
units of all ranks divided by the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), LBM_BENCH_BACKEND="gloo")
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    ms = 100.0 + 25.0 * rank  # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, w)
    out[rank] = (ms_max, bench.whole_job_mlups(w, 1_000_000, 10, ms_max))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0][0] == out[1][0] == 125.0
    # 2 replicas x 1e6 nodes x 10 steps in 125 ms
    assert out[0][1] == pytest.approx(2 * 1e6 * 10 / 0.125 / 1e6)
