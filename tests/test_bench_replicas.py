"""The multi-GPU bench path ("replicas only": every rank solves its own seeded geometry, no
collective on the data path) reduces its figures over the ranks: times by maximum, work by
sum.  Checked here on CPU with world size 2 over gloo."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times, units = bench.reduce_replicas(dist, "cpu", [1.0 + rank, 2.0, 3.0 * rank], 100 * (rank + 1))
    dist.destroy_process_group()
    out[rank] = (times, units)


def test_replica_reduction_two_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        for r in range(2):
            times, units = out[r]
            assert times == [2.0, 2.0, 3.0]
            assert units == 300.0


def test_replica_reduction_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_replicas(None, "cpu", [1.5, 2.5], 7) == ([1.5, 2.5], 7.0)
