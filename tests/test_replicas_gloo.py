"""The multi-GPU form of the benchmark is 'replicas only': independent
problems per rank, no collective on the data path, and the whole-job
throughput is all ranks' steps over the slowest rank's time.  This checks
that aggregation with two gloo ranks on the CPU."""

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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms = [1000.0, 2500.0][rank]
    v = bench.replica_throughput(steps=5, total_ms=total_ms, world=world)
    m = bench.max_over_ranks(total_ms, world)
    out[rank] = (v, m)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        v, m = res[rank]
        assert m == 2500.0
        assert abs(v - 2 * 5 / 2.5) < 1e-12


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_throughput(4, 2000.0, 1) == 2.0
