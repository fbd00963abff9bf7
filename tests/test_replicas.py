"""The multi-GPU form of the benchmark is replicas only (every solve is
independent, so nothing is exchanged on the data path): each rank times its
own solves and the job's time is the slowest rank's.  This checks that host
logic with two gloo ranks on the CPU (the same all_reduce(MAX) the benchmark
issues over NCCL)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]  # rank 1 is the slower replica
    total = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    out[rank] = (total, bench.replica_value(total, 10, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        total, value = res[rank]
        assert total == 150.0
        assert value == 150.0 / (10 * 2)


def test_single_process_value():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(42.0, None, None) == 42.0
    assert bench.replica_value(200.0, 20, 1) == 10.0
