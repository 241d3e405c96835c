"""The multi-GPU path of bench.py runs independent replicas (the step does
not shard); its host-side aggregation -- slowest rank's time, sum of the
ranks' work -- checked with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate_replicas(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world)
    q.put((rank, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, units in got:
        assert ms == 15.0          # the slowest rank
        assert units == 3000.0     # both ranks' work


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(7.0, 11.0, 1) == (7.0, 11.0)
