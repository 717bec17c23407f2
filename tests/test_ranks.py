"""The bench's multi-process aggregation on CPU (two gloo ranks).

With one process per GPU, each running a replica of the reconstruction, the job's time is
its slowest rank's and its work the sum of the ranks' patterns; every rank receives both."""
import os
import socket

import pytest

dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms, units = bench.over_ranks(dist, 10.0 + 5.0 * rank, 3600 * (rank + 1), "cpu")
        q.put((rank, ms, units))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_summed_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_rank, args=(world, _free_port(), q), nprocs=world, start_method="spawn", join=True)
    got = sorted(q.get() for _ in range(world))
    assert got == [(0, 15.0, 3600.0 * 3), (1, 15.0, 3600.0 * 3)]


def test_one_process_passes_through():
    import bench

    assert bench.over_ranks(None, 12.5, 7200, "cpu") == (12.5, 7200)
