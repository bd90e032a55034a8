"""The multi-rank bench path on CPU with gloo (world size 2): each rank
simulates its own bundle, and the job value sums node-updates over ranks and
divides by the slowest rank's time.  No GPU and no data-path collective."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.rank_workload(rank)
        local_updates = float(w.total_nodes) * 10
        local_seconds = 1.0 + rank  # rank 1 is the slow one
        total, tmax = bench.aggregate_over_ranks(local_updates, local_seconds, dist)
        q.put((rank, w.seed, w.total_nodes, total, tmax, int(w.mu_of_fiber.sum())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_aggregate_without_sharing_fibers():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, s0, n0, tot0, t0, mu0), (r1, s1, n1, tot1, t1, mu1) = res
    assert (s0, s1) == (5, 6)              # independent seeded bundles
    assert mu0 != mu1
    assert tot0 == tot1 == (n0 + n1) * 10.0  # node-updates summed over ranks
    assert t0 == t1 == 2.0                   # time of the slowest rank
