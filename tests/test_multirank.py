"""The N > 1 host logic of bench.py on CPU: two gloo ranks, each timing its
own replica, agree on the maximum over ranks and on the whole-job seconds
per solve."""
import os
import socket

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
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 + 50.0 * rank  # rank 1 is the slower replica
        out[rank] = bench.job_time(ms_local, 2, world, dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_replica():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (150.0, 75.0, 150.0 / 1000.0 / 4)


def test_one_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time(80.0, 4, 1) == (80.0, 20.0, 0.02)
