"""Replica path of bench.py on CPU: two gloo ranks agree on the slowest
rank's time, and each rank draws independent seeded inputs."""

import os

import numpy as np
import torch.multiprocessing as mp

import bench


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.reduce_max([1.5, 4.25][rank], world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = 29500 + os.getpid() % 1000
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == 4.25 and out[1] == 4.25


def test_replicas_get_independent_inputs():
    from workloads import small_target

    t = small_target(n_samples=1000, seed=5)
    a = bench.make_inputs(t, 0)
    b = bench.make_inputs(t, 1)
    assert not np.array_equal(a[0], b[0])
    assert np.array_equal(a[0], bench.make_inputs(t, 0)[0])
