"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the
barrier and the max/sum reductions used to combine per-rank timings.  The
data path has no collective: each rank checkpoints its own GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, _ = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    bench.barrier(dist)
    mx = bench.max_over_ranks(dist, 10.0 + r)
    sm = bench.sum_over_ranks(dist, 1.5 * (r + 1))
    out[r] = (r, w, mx, sm)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        rank, world, mx, sm = res[r]
        assert (rank, world) == (r, 2) and mx == 11.0 and sm == 4.5


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.0) == 3.0 and bench.sum_over_ranks(None, 2.0) == 2.0
