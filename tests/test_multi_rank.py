"""The N > 1 path of the benchmark on CPU: two `gloo` ranks, as torchrun would
start them.  Each rank takes its own slice of the sky lattice (weak scaling,
no data-path collective); the step time is the maximum over the ranks; the
job's rate counts every rank's units.  The per-sky top-k is complete on its
rank, so no result is exchanged."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import tcw_synth as syn  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, per_rank, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sky = bench.rank_sky(rank, world, per_rank)
        slices = [None] * world
        dist.all_gather_object(slices, sky)
        slow = bench.max_over_ranks(10.0 * (rank + 1), dist)     # rank r "took" 10 (r + 1) ms
        rate = bench.job_rate(world, 1000, 3, slow / 1000.0)
        dist.barrier()
        if rank == 0:
            out.put((slices, slow, rate))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_shard_the_sky_and_take_the_slowest_time(world):
    per_rank = 64
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, per_rank, out)) for r in range(world)]
    for p in procs:
        p.start()
    slices, slow, rate = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # disjoint slices whose union is the whole lattice, in rank order
    full = syn.fibonacci_sky(per_rank * world)
    np.testing.assert_array_equal(np.concatenate(slices), full)
    assert all(s.shape == (per_rank, 3) for s in slices)
    # the slowest rank sets the step time; every rank's units count
    assert slow == 10.0 * world
    assert rate == pytest.approx(world * 1000 * 3 / (slow / 1000.0))


def test_single_rank_helpers():
    assert bench.max_over_ranks(12.5) == 12.5
    np.testing.assert_array_equal(bench.rank_sky(0, 1, 32), syn.fibonacci_sky(32))
