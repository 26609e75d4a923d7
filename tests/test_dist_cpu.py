"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The layer shards by image: ranks never exchange data, only the timing
reduction (max over ranks) runs as a collective.  These tests run two gloo
ranks as processes and check the reduction, the image split and the
whole-job value.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [1.5, 2.25][rank]
    got = bench.max_over_ranks(ms, world, torch.device("cpu"))
    lo, hi = bench.shard(64, rank, world)
    bench.barrier(world)
    out[rank] = (got, lo, hi)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0][0] == 2.25 and out[1][0] == 2.25  # both ranks see the slowest time
    assert (out[0][1], out[0][2]) == (0, 32) and (out[1][1], out[1][2]) == (32, 64)


@pytest.mark.parametrize("n,world", [(64, 1), (64, 3), (5, 8), (0, 2)])
def test_shard_covers_every_image_once(n, world):
    seen = []
    for r in range(world):
        lo, hi = bench.shard(n, r, world)
        seen.extend(range(lo, hi))
    assert seen == list(range(n))


def test_job_value_is_all_pixels_over_slowest_rank():
    assert bench.job_value(4 * 2048 * 2048, 2, 1.0) == pytest.approx(2 * 4 * 2048 * 2048 / 1e-3 / 1e6)
