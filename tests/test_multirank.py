"""The N > 1 path of bench.py (independent replicas, max-over-ranks timing) with gloo on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 * (rank + 1)  # rank 1 is the slow one
    ms_max, value = bench.aggregate(ms_local, world, units_per_rank=1000, steps=5)
    out[rank] = (ms_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_max_time_and_report_the_whole_job_rate():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms_max, value = out[r]
        assert ms_max == pytest.approx(20.0)
        assert value == pytest.approx(world * 1000 * 5 / 20e-3)


def test_single_rank_needs_no_process_group():
    import bench
    ms, v = bench.aggregate(4.0, 1, 100, 10)
    assert ms == 4.0 and v == pytest.approx(100 * 10 / 4e-3)
