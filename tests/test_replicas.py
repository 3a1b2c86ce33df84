"""The N > 1 path of bench.py (independent replicas, no data-path collective): with two gloo
ranks on the CPU every rank receives the slowest rank's time, and the reported rate is all
ranks' particles over that time."""
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
    local_ms = [120.0, 150.0][rank]
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    out[rank] = (ms, bench.replica_throughput(1_000_000, 10, world, ms))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert res[0][1] == pytest.approx(2 * 1_000_000 * 10 / 0.150)
    assert res[0][1] == res[1][1]


def test_single_rank_is_plain():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.replica_throughput(10, 2, 1, 1000.0) == 20.0
