"""Multi-process path of bench.py on CPU (gloo, world size 2): the lattice
problem does not shard, so N GPUs run N replicas; the reported throughput is
the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.replica_aggregate(dist, elapsed_ms=100.0 + 50.0 * rank, units=1e9 * (rank + 1))
    out.put((rank, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, units in res:
        assert ms == 150.0            # max over ranks
        assert units == 3e9           # sum over ranks


def test_replica_aggregation_single_process():
    import bench
    assert bench.replica_aggregate(None, 12.0, 5.0) == (12.0, 5.0)
