"""The multi-process path of bench.py on CPU: two gloo ranks, each with its
own replica, combine their timings as the benchmark does (max over ranks,
whole-job throughput = all ranks' particle-steps / slowest rank's time)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [0.25, 0.5][rank]           # per-rank timed region
        worst = bench.combine_ranks(secs, world)
        n_per_rank, steps = 1000, 10
        value = bench.job_throughput(n_per_rank, world, steps, worst)
        out[rank] = (worst, value)
        bench._barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench():
    world = 2
    mgr = mp.get_context("spawn").Manager()  # no fork: earlier tests may have started threads
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    worst, value = out[0]
    assert worst == 0.5
    assert value == pytest.approx(2 * 1000 * 10 / 0.5)
