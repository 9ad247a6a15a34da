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


class _FakeImage:
    def __init__(self, seq):
        self.seq = seq

    def info(self):
        return {"seq": self.seq}


class _FakeSet:
    """Host stand-in for a rank's CheckpointSet (the cut logic is host-only)."""

    def __init__(self, skip_first=False):
        self.seq = 1 if skip_first else 0
        self.restored = None

    def checkpoint(self, stream, flags=0):
        img = _FakeImage(self.seq)
        self.seq += 1
        return img

    def restore(self, image, stream):
        self.restored = image.seq


def _cut_worker(rank, world, port, out, skew):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1808_00117_b300 import cut
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    s = _FakeSet(skip_first=skew and rank == 1)
    res = []
    for _ in range(2):
        try:
            img, c = cut.checkpoint_cut(s, 0)
            res.append(("ok", c))
        except cut.CutError as e:
            res.append(("refused", str(e)))
    try:
        res.append(("restored", cut.restore_cut(s, _FakeImage(0), 0), s.restored))
    except cut.CutError:
        res.append(("restore refused",))
    out[rank] = res
    dist.destroy_process_group()


@pytest.mark.parametrize("skew", [False, True])
def test_consistent_cut_two_ranks(skew):
    """In step, both ranks agree on cuts 0 and 1 and restore cut 0; a rank
    that is one checkpoint ahead makes every rank refuse each cut."""
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_cut_worker, args=(2, port, out, skew), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        if not skew:
            assert res[r] == [("ok", 0), ("ok", 1), ("restored", 0, 0)]
        else:
            assert [x[0] for x in res[r][:2]] == ["refused", "refused"]
            assert res[r][2] == ("restored", 0, 0)
