"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every
rank gets its own load scenario of the same grid, and the job's numbers are
the slowest rank's time and the sums of solves and iterations."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    g = bench.replica_grid(rank, world)
    # rank r reports (time 1 + r, converged 3 + r, iterations 100 r)
    out = bench.combine_ranks(1.0 + rank, 3 + rank, 100 * rank, world, torch.device("cpu"))
    q.put((rank, out, float(g.pd.sum()), g.nbus))
    dist.destroy_process_group()


def test_two_rank_replicas_and_totals():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, out, _, nb in res:
        assert out == (2.0, 7, 100)  # max time, summed solves and iterations
        assert nb == 2000
    # distinct scenarios per rank
    assert abs(res[0][2] - res[1][2]) > 1e-6
