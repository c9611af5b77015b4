"""The N > 1 path of the benchmark on CPU: two gloo ranks (127.0.0.1), each timing its
own replica; the job time is the slowest rank's and the rate counts every rank's units.
The reference arm runs on rank 0 only (the other ranks return nothing)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(torch, ms, world, "cpu")
        rate = bench.whole_job_rate(1_000_000, world, ms_max)
        ref = bench.run_reference(_Args(), rank, world) if rank == 1 else None
        q.put((rank, ms_max, rate, ref))
    finally:
        dist.destroy_process_group()


class _Args:
    steps, warmup, n3, n2 = 1, 0, 512, 16384


def test_two_gloo_ranks_take_the_max_and_count_all_units():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, ms_max, rate, ref = q.get(timeout=120)
        out[rank] = (ms_max, rate, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        assert out[rank][0] == 150.0  # the slowest rank on every rank
        assert out[rank][1] == pytest.approx(2 * 1_000_000 / 0.150 / 1e6)
    assert out[1][2] is None  # the reference arm runs on rank 0 only


def test_single_rank_is_identity():
    assert bench.max_over_ranks(torch, 12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(3_000_000, 1, 1000.0) == pytest.approx(3.0)
