"""The N > 1 path of bench.py (independent replicas, one per rank; the job's time is
the slowest rank's) on two gloo ranks on the host. CPU only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_init()
        ms = 100.0 * (rank + 1)  # rank 1 is the slow replica
        slow = bench.max_over_ranks(ms)
        out[rank] = (w, r, loc, slow, bench.replica_throughput(w, 5, slow))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, loc, slow, value = res[rank]
        assert (w, r, loc) == (world, rank, rank)
        assert slow == 200.0  # every rank sees the slowest replica's time
        assert value == pytest.approx(world * 5 / 0.2)  # units of all ranks over that time


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_throughput(1, 4, 2000.0) == pytest.approx(2.0)
