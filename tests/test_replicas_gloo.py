"""The N > 1 path of bench.py (independent replicas, no data-path collective): two gloo ranks on the
CPU gather their per-rank figures; the job time is the slowest rank's, bytes and itemsets add up."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.5 + rank, 1000.0 * (rank + 1), 10 + rank, 0.25 * (rank + 1)]
        allv = bench.gather_ranks(mine, dist, world, "cpu")
        q.put((rank, allv.tolist(), bench.combine_ranks(allv)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_combine():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, allv, comb in out:
        assert np.allclose(allv, [[1.5, 1000.0, 10, 0.25], [2.5, 2000.0, 11, 0.5]])
        assert comb == (2.5, 3000.0, 21.0, 0.5)


def test_single_rank_is_one_row():
    sys.path.insert(0, ROOT)
    import bench

    allv = bench.gather_ranks([3.0, 4.0, 5.0, 6.0], None, 1, "cpu")
    assert allv.shape == (1, 4) and bench.combine_ranks(allv) == (3.0, 4.0, 5.0, 6.0)
