"""The multi-rank (replica) reduction of bench.py on CPU: two gloo ranks with
different step times must both report the slower rank's time and the
whole-job rate world * 1000 / t_max."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t_max, rate = bench.replica_rate(1.5 + rank, world, "cpu")
        out[rank] = (t_max, rate)
    finally:
        dist.destroy_process_group()


def test_replica_rate_takes_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.5, world * 1000.0 / 2.5)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.replica_rate(4.0, 1) == (4.0, 250.0)
