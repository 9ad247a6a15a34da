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
    with mp.get_context("spawn").Manager() as m:  # no fork of a CUDA process
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        rank, world, mx, sm = res[r]
        assert (rank, world) == (r, 2) and mx == 11.0 and sm == 4.5


def test_host_budget_is_shared_by_the_ranks_of_a_node(monkeypatch):
    # each rank pins images in its share of the node's available memory
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("LOCAL_WORLD_SIZE", "1")
    one = bench.host_budget_bytes()
    monkeypatch.setenv("LOCAL_WORLD_SIZE", "4")
    four = bench.host_budget_bytes()
    assert one > 0 and abs(4 * four - one) <= 0.05 * one  # available memory moves a little


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.0) == 3.0 and bench.sum_over_ranks(None, 2.0) == 2.0


class _FakeImage:
    def __init__(self, seq):
        self.seq = seq
        self.released = False

    def info(self):
        return {"seq": self.seq}

    def release(self):
        self.released = True


class _FakeSet:
    """Host stand-in for a rank's CheckpointSet (the cut logic is host-only)."""

    def __init__(self, fail_at=()):
        self.seq = 0
        self.calls = 0
        self.fail_at = set(fail_at)
        self.restored = None
        self.taken = []

    def checkpoint(self, stream, flags=0):
        self.calls += 1
        if self.calls in self.fail_at:
            raise RuntimeError("injected checkpoint failure")
        img = _FakeImage(self.seq)
        self.taken.append(img)
        self.seq += 1
        return img

    def restore(self, image, stream):
        self.restored = image.seq


def _cut_worker(rank, world, port, out, mode):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1808_00117_b300 import cut
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    # "skew": rank 1 believes it is one cut ahead; "fail": rank 1's second
    # checkpoint raises
    s = _FakeSet(fail_at=(2,) if mode == "fail" and rank == 1 else ())
    co = cut.CutCoordinator(s, first_cut=1 if mode == "skew" and rank == 1 else 0)
    res = []
    for _ in range(3):
        try:
            img, c = co.checkpoint(0)
            res.append(("ok", c, img.seq))
        except cut.CutError:
            res.append(("refused",))
    res.append(("released", [img.released for img in s.taken]))
    ok_cuts = sorted(co.images)
    for c in (ok_cuts[0], 99):
        try:
            res.append(("restored", co.restore(c, 0), s.restored))
        except cut.CutError:
            res.append(("restore refused", c))
    res.append(("seqs", {k: v for k, v in co.seqs.items()}))
    out[rank] = res
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["in_step", "skew", "fail"])
def test_consistent_cut_two_ranks(mode):
    """In step: cuts 0, 1, 2 stand on both ranks.  Skew (rank 1 one cut
    ahead): the first cut is refused on both ranks, each drops the image it
    took, and both continue in step from cut 2.  Fail (rank 1's second
    checkpoint raises): that cut is refused on both ranks, the rank that did
    capture drops its image, and the next cut stands.  A restore of a cut
    every rank holds runs everywhere; of one nobody holds, is refused
    everywhere."""
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a CUDA process
        out = m.dict()
        mp.spawn(_cut_worker, args=(2, port, out, mode), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        got = res[r]
        if mode == "in_step":
            assert got[:3] == [("ok", 0, 0), ("ok", 1, 1), ("ok", 2, 2)]
            assert got[3] == ("released", [False, False, False])
            assert got[4] == ("restored", 0, 0)
        elif mode == "skew":
            assert got[:3] == [("refused",), ("ok", 2, 1), ("ok", 3, 2)]
            assert got[3] == ("released", [True, False, False])
            assert got[4] == ("restored", 2, 1)
            assert got[6] == ("seqs", {2: [1, 1], 3: [2, 2]})
        else:
            assert got[0] == ("ok", 0, 0) and got[1] == ("refused",)
            # rank 0 captured at the refused cut; its image stays in its
            # chain, so its sequence number runs one ahead of rank 1's
            assert got[2] == ("ok", 2, 2 if r == 0 else 1)
            assert got[3] == ("released", [False, True, False] if r == 0 else [False, False])
            assert got[6] == ("seqs", {0: [0, 0], 2: [2, 1]})
        assert got[5] == ("restore refused", 99)


def _lost_worker(rank, world, port, out):
    import datetime
    import sys
    import time
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1808_00117_b300 import cut
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=20))
    s = _FakeSet()
    co = cut.CutCoordinator(s, timeout_s=3.0)
    res = []
    img, c = co.checkpoint(0)
    res.append(("ok", c))
    if rank == 1:
        out[rank] = res  # rank 1 leaves between cuts, without a word
        return
    t0 = time.time()
    try:
        co.checkpoint(0)
        res.append(("ok",))
    except cut.RankLost:
        res.append(("lost", time.time() - t0 < 15))
    res.append(("released", [im.released for im in s.taken]))
    out[rank] = res


def test_cut_detects_a_rank_that_left():
    """Failure detection on the host: rank 1 takes cut 0 and exits; rank 0's
    next cut raises RankLost within the coordinator's timeout instead of
    waiting for ever, having queued no capture for it."""
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_lost_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[1] == [("ok", 0)]
    assert res[0][0] == ("ok", 0)
    assert res[0][1] == ("lost", True)
    assert res[0][2] == ("released", [False])  # no image was taken for the lost cut
