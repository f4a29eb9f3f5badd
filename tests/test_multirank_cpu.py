"""Multi-rank path of the benchmark on CPU (gloo, world size 2).

The flood pipeline runs as independent replicas (one cloud per GPU, no
collective on the data path); the only exchange is the job-level timing: the
slowest rank's step time and the sum of every rank's units.
"""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate(10.0 + 5.0 * rank, 1000.0 * (rank + 1))
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_aggregate_takes_slowest_rank_and_sums_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(12.5, 77.0) == (12.5, 77.0)
