"""The N > 1 host path of bench.py on CPU: two gloo ranks.

Under torchrun every rank filters its own image (independent problems, no
collective on the data path); the job's time is the slowest rank's, and the
throughput counts every rank's pixels.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        total = bench.reduce_max(local_ms, dist, "cpu")
        img = bench.make_input("rects4096-crop", 64, 64, rank)
        digest = float(np.asarray(img, dtype=np.float64).sum())
        t = torch.tensor([digest], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, t)
        out[rank] = (total, [float(g.item()) for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_filter_distinct_images():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 15.0
    digests = out[0][1]
    assert digests == out[1][1]
    assert digests[0] != digests[1]  # each rank has its own seeded image


def test_job_throughput_counts_every_rank():
    # 4 ranks x 2 steps x 1 Mpx in 1 s of the slowest rank
    assert bench.job_throughput(1_000_000, 4, 2, 1000.0) == pytest.approx(8.0)
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
