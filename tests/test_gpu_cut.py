"""Consistent cut on real checkpoint sets (Section 3.3 / 4.5: every rank
quiesces, then checkpoints).  Two ranks, spawned as processes that share
the one GPU, each with its own CheckpointSet over its own seeded device
buffers and its own oracle; the cut protocol runs over gloo on the host.
The ranks' kernels never wait on one another: each rank's capture and
restore are its own stream-ordered work, and all coordination is host
barriers and all-gathers.

Every image a rank takes at a cut that stands equals its oracle's image
byte for byte; a cut that one rank cannot take (its checkpoint call fails)
or that finds a rank out of step is refused on both ranks and the protocol
continues in step; restoring a cut onto scribbled memory gives back each
rank's state at that cut, and a restore of a refused cut is refused."""
import os
import socket

import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = 65536


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out, mode):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    import paper_1808_00117_b300 as crum
    from paper_1808_00117_b300 import cut
    from paper_1808_00117_b300 import workloads as W

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    torch.cuda.set_device(0)
    crum.load()
    sizes = [5 * P + 4104 * (rank + 1), 12 * P + 8, 3 * P]
    bufs = []
    for i, n in enumerate(sizes):
        b = torch.empty(n, dtype=torch.uint8, device="cuda")
        W.fill_(b, 9100 + 10 * rank + i, ["u32", "fp32", "fp64"][i])
        bufs.append(b)
    torch.cuda.synchronize()
    s = crum.CheckpointSet()
    for b in bufs:
        s.register(b.data_ptr(), b.numel())
    o = oracle.OracleSet(sizes)
    co = cut.CutCoordinator(s, first_cut=1 if mode == "skew" and rank == 1 else 0)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def host():
        stream.synchronize()
        return [b.cpu().numpy().copy() for b in bufs]

    res, states, errors = [], {}, []
    for step in range(4):
        if step:
            for i, b in enumerate(bufs):
                n = W.pages_of(sizes[i])
                W.mutate_pages_(b, W.choose_uniform(300 * rank + 10 * step + i, n, max(1, n // 3)),
                                500 * rank + 10 * step + i)
        # "fail": rank 1's checkpoint call at step 2 fails (verify-mode flag
        # on a set made without verify: EINVAL before any device work)
        flags = crum.VERIFY if mode == "fail" and rank == 1 and step == 2 else crum.INCR
        try:
            img, c = co.checkpoint(sh, flags)
            img.wait()
            state = host()
            exp, *_ = o.checkpoint(state)
            if img.to_bytes() != exp:
                errors.append(f"image of cut {c} differs from the oracle's")
            states[c] = state
            res.append(("ok", c))
        except cut.CutError:
            res.append(("refused",))
            if flags == crum.INCR:
                # this rank's capture ran: its image is a link of its chain,
                # so the oracle takes the same checkpoint
                o.checkpoint(host())
    for c in sorted(states):
        for i, b in enumerate(bufs):
            W.fill_(b, 777 + c + i, "u32")
        co.restore(c, sh, wait=stream.synchronize)
        if any(not np.array_equal(g, e) for g, e in zip(host(), states[c])):
            errors.append(f"restore of cut {c} differs from the state at that cut")
    refused = [k for k in range(4) if k not in states]
    try:
        co.restore(refused[0] if refused else 99, sh)
        res.append(("restore of a refused cut ran",))
    except cut.CutError:
        res.append(("restore refused",))
    co.release()
    s.destroy()
    out[rank] = {"res": res, "errors": errors, "seqs": dict(co.seqs)}
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["in_step", "fail", "skew"])
def test_cut_on_two_ranks_sharing_the_gpu(mode):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a CUDA process
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out, mode), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        assert res[r]["errors"] == [], res[r]["errors"]
        got = res[r]["res"]
        if mode == "in_step":
            assert got == [("ok", 0), ("ok", 1), ("ok", 2), ("ok", 3), ("restore refused",)]
            assert res[r]["seqs"] == {k: [k, k] for k in range(4)}
        elif mode == "fail":
            assert got == [("ok", 0), ("ok", 1), ("refused",), ("ok", 3), ("restore refused",)]
            # rank 0 captured at the refused cut, so its sequence runs ahead
            assert res[r]["seqs"][3] == [3, 2]
        else:
            assert got == [("refused",), ("ok", 2), ("ok", 3), ("ok", 4), ("restore refused",)]
            assert res[r]["seqs"][2] == [1, 1]
