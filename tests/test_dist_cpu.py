"""Multi-rank path of the benchmark on CPU (gloo, world size 2).

The filter-and-mix path has no exchange step: N GPUs run N replicas and the
benchmark only aggregates time (max over ranks) and units (sum over ranks).
"""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(10.0 + 5.0 * rank, dist)       # rank 1 is slower
    rate = bench.whole_job_rate(100.0, world, ms)
    dist.barrier()
    q.put((rank, ms, rate))
    dist.destroy_process_group()


def test_replica_timing_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 15.0                                   # the slowest rank's time
        assert abs(rate - 2 * 100.0 / 0.015) < 1e-6        # both replicas' units
