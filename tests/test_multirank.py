"""The bench's multi-rank aggregation on world_size 2 with gloo on CPU: every
rank advances its own replica, the job time is the slowest rank's, and the
throughput counts every rank's cells."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 * (rank + 1)        # rank 1 is the slower one
        ms = bench.max_over_ranks(ms_local, dist, "cpu")
        out[rank] = (ms, bench.job_mlups(1000, 50, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_with_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, mlups = res[r]
        assert ms == 20.0
        assert mlups == pytest.approx(2 * 1000 * 50 / 0.020 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_mlups(100, 10, 1, 1.0) == pytest.approx(1.0)


def test_rev_library_slices_are_disjoint_and_reproducible():
    """Each rank of the REV workload advances its own runs of one seeded
    library: the slices cover the library without overlap, and a run is the
    same REV whichever slice generates it."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    world, per = 3, 2
    slices = [bench.rev_slice(per, r) for r in range(world)]
    covered = sorted(i for first, n in slices for i in range(first, first + n))
    assert covered == list(range(world * per))
    seed = 12345
    whole = bench.rev_library(4, seed)
    part = bench.rev_library(2, seed, first=2)
    for (e1, k1, c1, p1), (e2, k2, c2, p2) in zip(whole[2:], part):
        assert (e1, k1) == (e2, k2)
        np.testing.assert_array_equal(c1, c2)
        np.testing.assert_array_equal(p1, p2)
