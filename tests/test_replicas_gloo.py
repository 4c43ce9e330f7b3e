"""Multi-GPU replicas (the filter needs no exchange between GPUs): the
host-side bookkeeping bench.py uses under torchrun -- max-over-ranks timing,
whole-job throughput, distinct inputs per rank and gathering the ranks'
results -- with two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slower replica
        ms = bench.max_over_ranks(local_ms, torch.device("cpu"))
        v = bench.job_throughput(world, 1920 * 1080, 100, ms)
        q.put((rank, ms, v))
    finally:
        dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_pixels():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, v in res:
        assert ms == pytest.approx(15.0)
        assert v == pytest.approx(2 * 1920 * 1080 * 100 / 0.015 / 1e6)


def _filter_rank(rank, world, port, q):
    """One replica: draw this rank's own inputs (bench's seed rule), filter a
    crop of them -- with the CPU oracle, the GPU filter's stand-in on a
    machine without a GPU -- and gather every rank's result on rank 0."""
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1811_02308_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.replica_seed(rank, 0)
        f, th, s = synth.make_inputs(48, 64, seed, n_blobs=4, zeta_range=(-20, 20), sigma_range=(5, 60))
        g, _ = oracle.fabf(f, th, s, 5, 5)
        got = [None] * world
        dist.all_gather_object(got, (rank, seed, g))
        if rank == 0:
            q.put(got)
    finally:
        dist.destroy_process_group()


def test_replicas_filter_their_own_images_and_gather(oracle_mod):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_filter_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_1811_02308_gb300 import synth
    assert [r for r, _, _ in got] == [0, 1]
    assert got[0][1] != got[1][1]                     # distinct inputs per replica
    assert not np.array_equal(got[0][2], got[1][2])
    for rank, seed, g in got:                          # each result is its own image's
        f, th, s = synth.make_inputs(48, 64, seed, n_blobs=4, zeta_range=(-20, 20), sigma_range=(5, 60))
        ref, _ = oracle_mod.fabf(f, th, s, 5, 5)
        assert np.array_equal(g, ref)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import torch

    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.job_throughput(1, 1000, 10, 1.0) == pytest.approx(10.0)
