"""The multi-GPU path is replicas only: each rank answers its own copy of the
query batch and the job's throughput is all ranks' queries over the slowest
rank's time.  This checks bench.py's aggregation with two gloo ranks on CPU
(no GPU; the GPU run uses the same function over NCCL)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.replica_throughput(local_ms[rank], 1000, world, dist, "cpu")
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    local_ms = [40.0, 50.0]
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), local_ms, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 50.0
        assert abs(value - 2 * 1000 / 0.050) < 1e-6


def test_single_rank_is_its_own_time():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ms, value = bench.replica_throughput(25.0, 500, 1)
    assert ms == 25.0 and abs(value - 500 / 0.025) < 1e-9
