"""Serving: checkpoint/restore requests from several clients through
crum_server, several on the device at once.  Each client's results must be
the same alone and in the mix (exact: integer work), and equal the oracle's
images; admission must respect the staging budget."""
import numpy as np
import pytest

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W

from helpers import torch

pytestmark = pytest.mark.gpu
P = 65536
SIZES = [3 * P + 5, 40 * P, 7 * P + 100, 16 * P]


@pytest.fixture(autouse=True)
def _cuda():
    if not torch().cuda.is_available():
        pytest.skip("needs a CUDA device")
    crum.load()


class Client:
    def __init__(self, server, idx, size, restore_mode=crum.RESTORE_AUTO, memory="device"):
        t = torch()
        self.idx, self.size = idx, size
        self.stream = t.cuda.Stream()
        # device memory, managed memory on the device, or managed memory the
        # client keeps in host memory (read in place by its set)
        if memory == "device":
            self.buf = t.empty(size, dtype=t.uint8, device="cuda")
        else:
            self.buf = W.managed_empty(size)
        W.fill_(self.buf, 600 + idx, "fp32")
        t.cuda.synchronize()
        if memory == "host_managed":
            W.managed_prefetch(self.buf.data_ptr(), size, "host")
        self.set = crum.CheckpointSet(external_staging=1, restore_mode=restore_mode,
                                      managed_in_place=int(memory == "host_managed"))
        self.set.register(self.buf.data_ptr(), size)
        self.cid = server.add_client(self.set, self.stream.cuda_stream)
        self.restore_mode = restore_mode
        self.oracle = oracle.OracleSet([size])
        self.step = 0
        self.states = []

    def host(self):
        self.stream.synchronize()
        return self.buf.cpu().numpy().copy()

    def mutate(self):
        self.step += 1
        n = W.pages_of(self.size)
        pages = W.choose_uniform(self.idx * 1000 + self.step, n, max(1, n // 3))
        with torch().cuda.stream(self.stream):
            W.mutate_pages_(self.buf, pages, self.idx * 77 + self.step)


def run_sequence(server, clients, rounds, restore_at):
    """Each round: every client mutates and submits a checkpoint; the
    client waits for its capture before touching its memory again.  At
    round `restore_at` every client also asks for a restore.  Returns per
    client the checksums of its checkpoint images and the oracle's."""
    got = {c.idx: [] for c in clients}
    exp = {c.idx: [] for c in clients}
    pending = []
    for rnd in range(rounds):
        round_ids = []
        for c in clients:
            if rnd:
                c.mutate()
            round_ids.append((c, server.submit(c.cid, crum.REQ_CHECKPOINT)))
        for c, rid in round_ids:
            server.wait(rid, crum.WAIT_CAPTURED)
            state = c.host()
            c.states.append(state)
            img, *_ = c.oracle.checkpoint([state])
            exp[c.idx].append(int(np.frombuffer(img[-8:], dtype=np.uint64)[0]))
            pending.append((c, rid))
        if rnd == restore_at:
            for c in clients:
                # scribble (all of it, or a third of the pages for a delta
                # restore), then restore the newest chain: memory must come back
                if c.restore_mode == crum.RESTORE_DELTA:
                    c.mutate()
                else:
                    with torch().cuda.stream(c.stream):
                        W.fill_(c.buf, 999, "u32")
                rid = server.submit(c.cid, crum.REQ_RESTORE)
                info = server.wait(rid)
                assert info["done"] and info["status"] == crum.OK
                assert np.array_equal(c.host(), c.states[-1])
    for c, rid in pending:
        info = server.wait(rid)
        assert info["status"] == crum.OK
        got[c.idx].append(info["checksum"])
    return got, exp


@pytest.mark.parametrize("lanes,mode,serial", [((-1, -1), crum.RESTORE_AUTO, -1),
                                               ((1, 1), crum.RESTORE_AUTO, -1),
                                               ((1, 1), crum.RESTORE_DELTA, -1),
                                               ((3, 1), crum.RESTORE_DELTA, 1),
                                               ((0, 0), crum.RESTORE_AUTO, 0)])
def test_same_alone_and_in_the_mix(lanes, mode, serial):
    srv = crum.Server(staging_budget=1 << 30, max_inflight=3, max_checkpoints=lanes[0],
                      max_restores=lanes[1], serialize_drains=serial)
    mix = [Client(srv, i, s, mode) for i, s in enumerate(SIZES)]
    got_mix, exp = run_sequence(srv, mix, rounds=4, restore_at=2)
    stats = srv.drain()
    assert stats["failed"] == 0 and stats["completed"] == 4 * len(SIZES) + len(SIZES)
    if lanes[0] < 0:
        assert stats["peak_inflight"] >= 2  # requests of different clients overlapped
    for i in range(len(SIZES)):
        assert got_mix[i] == exp[i], f"client {i} in the mix differs from the oracle"
    srv.destroy()
    # each client alone, same seeds: same images
    for i, s in enumerate(SIZES):
        srv1 = crum.Server(staging_budget=1 << 30, max_inflight=3, serialize_drains=serial)
        alone = Client(srv1, i, s, mode)
        got_alone, _ = run_sequence(srv1, [alone], rounds=4, restore_at=2)
        assert got_alone[i] == got_mix[i], f"client {i} alone differs from the mix"
        srv1.destroy()


def test_admission_respects_the_budget():
    # budget holds the 40-page client or two small ones, never all at once
    budget = 48 * P
    srv = crum.Server(staging_budget=budget, max_inflight=8, max_checkpoints=-1, max_restores=-1)
    clients = [Client(srv, 10 + i, s) for i, s in enumerate(SIZES)]
    ids = []
    for rnd in range(3):
        for c in clients:
            if rnd:
                c.mutate()
            ids.append(srv.submit(c.cid, crum.REQ_CHECKPOINT_FULL if rnd == 0 else crum.REQ_CHECKPOINT))
            srv.wait(ids[-1], crum.WAIT_CAPTURED)
    stats = srv.drain()
    assert stats["failed"] == 0 and stats["completed"] == len(ids)
    assert stats["peak_staging"] <= budget
    srv.destroy()


def test_client_larger_than_budget_is_rejected():
    srv = crum.Server(staging_budget=4 * P, max_inflight=2)
    t = torch()
    buf = t.empty(8 * P, dtype=t.uint8, device="cuda")
    s = crum.CheckpointSet(external_staging=1)
    s.register(buf.data_ptr(), buf.numel())
    with pytest.raises(crum.CrumError) as e:
        srv.add_client(s, t.cuda.current_stream().cuda_stream)
    assert e.value.status == crum.EINVAL
    srv.destroy()


def test_managed_clients_in_the_mix():
    """Clients whose memory is managed, on the device or kept in host memory
    (read in place), served together with a device-memory client: every
    image equals the oracle's and every restore brings the memory back."""
    srv = crum.Server(staging_budget=1 << 30, max_inflight=4, max_checkpoints=-1, max_restores=-1)
    kinds = ["device", "managed", "host_managed", "host_managed"]
    mix = [Client(srv, 20 + i, s, crum.RESTORE_AUTO, kinds[i]) for i, s in enumerate(SIZES)]
    got, exp = run_sequence(srv, mix, rounds=4, restore_at=2)
    stats = srv.drain()
    assert stats["failed"] == 0
    for c in mix:
        assert got[c.idx] == exp[c.idx], f"client {c.idx} ({kinds[c.idx - 20]}) differs from the oracle"
    srv.destroy()


# The serving configuration's request mix, scaled to a test: 8 clients with
# footprints log-uniform 1 MiB..1 GiB (4 KiB granularity, so tail pages are
# partial; 1.32 GiB in all, the largest 781 MiB), int32/fp32/fp64 data in
# turn, each request preceded by a rewrite of U[1 %, 50 %] of the client's
# pages, 80 % checkpoints (every fourth of a client full) and 20 % restores
# (a restore rolls the rewrite back).
MIX_SEED = 0x5EED + 30
MIX_KINDS = ["u32", "fp32", "fp64"]


class MixClient:
    def __init__(self, server, idx, size):
        t = torch()
        self.idx, self.size = idx, size
        self.pages = W.pages_of(size)
        self.stream = t.cuda.Stream()
        self.buf = t.empty(size, dtype=t.uint8, device="cuda")
        W.fill_(self.buf, 6100 + idx, MIX_KINDS[idx % 3])
        t.cuda.synchronize()
        self.set = crum.CheckpointSet(external_staging=1, restore_mode=crum.RESTORE_DELTA)
        self.set.register(self.buf.data_ptr(), size)
        self.cid = server.add_client(self.set, self.stream.cuda_stream)
        self.oracle = oracle.OracleSet([size])
        self.n_ckpt = 0
        self.state = None

    def host(self):
        self.stream.synchronize()
        return self.buf.cpu().numpy().copy()

    def rewrite(self, rnd, frac):
        k = max(1, int(round(frac * self.pages)))
        pages = W.choose_uniform(MIX_SEED + 97 * rnd + self.idx, self.pages, k)
        with torch().cuda.stream(self.stream):
            W.mutate_pages_(self.buf, pages, MIX_SEED + 131 * rnd + self.idx)


def run_mix(server, clients, rounds, plan):
    """Every round each client rewrites its share of pages and submits its
    request of that round (they run on the device together).  A checkpoint
    request's image, taken from the server, must equal the oracle's image of
    the client's memory at its capture, byte for byte; a restore must bring
    back the memory of the client's newest checkpoint.  Returns the SHA-256
    of every image, per client."""
    import hashlib
    digests = {c.idx: [] for c in clients}
    for rnd in range(rounds):
        ids = []
        for c in clients:
            restore, frac = plan[c.idx][rnd]
            if rnd:
                c.rewrite(rnd, frac)
            if restore:
                kind = crum.REQ_RESTORE
            else:
                kind = crum.REQ_CHECKPOINT_FULL if c.n_ckpt % 4 == 0 else crum.REQ_CHECKPOINT
                c.n_ckpt += 1
            ids.append((c, kind, server.submit(c.cid, kind)))
        for c, kind, rid in ids:
            if kind == crum.REQ_RESTORE:
                info = server.wait(rid)
                assert info["status"] == crum.OK
                assert np.array_equal(c.host(), c.state), f"client {c.idx} restore, round {rnd}"
                continue
            server.wait(rid, crum.WAIT_CAPTURED)
            c.state = c.host()
            exp, *_ = c.oracle.checkpoint([c.state], full=kind == crum.REQ_CHECKPOINT_FULL)
            info = server.wait(rid)
            assert info["status"] == crum.OK and info["checksum"] == int.from_bytes(exp[-8:], "little")
            img = server.take_image(rid)
            got = img.to_bytes()
            img.release()
            assert got == exp, f"client {c.idx} round {rnd}: image differs from the oracle's"
            digests[c.idx].append(hashlib.sha256(got).hexdigest())
    return digests


def mix_plan(sizes, rounds):
    rng = np.random.default_rng(MIX_SEED)
    plan = {}
    for i in range(len(sizes)):
        restore = rng.random(rounds) < 0.2
        restore[0] = False  # a client's first request is a checkpoint
        plan[i] = [(bool(r), float(f)) for r, f in zip(restore, rng.uniform(0.01, 0.50, rounds))]
    return plan


@pytest.mark.parametrize("lanes,serial,order", [((0, 0), 0, 0), ((-1, -1), -1, 0), ((2, 1), -1, 1)],
                         ids=["default_lanes", "unrestricted", "size_first"])
def test_config_mix_images_equal_the_oracle_alone_and_in_the_mix(lanes, serial, order):
    """The scaled serving mix under a 1.5 GiB staging budget: GiB-sized
    staging regions, the drain sequencer and long drains.  Every checkpoint
    image equals the oracle's byte for byte in the mix, and each client run
    alone through its own server gives the same images."""
    sizes = W.loguniform_sizes(MIX_SEED, 8, W.MiB, W.GiB, None, round_to=4096)
    rounds = 6
    plan = mix_plan(sizes, rounds)
    budget = 3 << 29
    srv = crum.Server(staging_budget=budget, max_inflight=8, max_checkpoints=lanes[0],
                      max_restores=lanes[1], serialize_drains=serial, keep_images=1, order=order)
    mix = [MixClient(srv, i, s) for i, s in enumerate(sizes)]
    in_mix = run_mix(srv, mix, rounds, plan)
    stats = srv.drain()
    assert stats["failed"] == 0 and stats["completed"] == rounds * len(sizes)
    assert stats["peak_staging"] <= budget and stats["peak_inflight"] >= 2
    srv.destroy()
    for c in mix:
        c.set.destroy()
    del mix
    for i, s in enumerate(sizes):
        srv1 = crum.Server(staging_budget=budget, max_inflight=8, keep_images=1)
        alone = MixClient(srv1, i, s)
        got = run_mix(srv1, [alone], rounds, plan)
        assert got[i] == in_mix[i], f"client {i} alone differs from the mix"
        srv1.destroy()
        alone.set.destroy()


def test_take_image_rules():
    """take_image: only with keep_images, only for a finished checkpoint
    request, and only once."""
    srv = crum.Server(staging_budget=1 << 28, max_inflight=2, keep_images=1)
    c = MixClient(srv, 0, 3 * P + 4096)
    rid = srv.submit(c.cid, crum.REQ_CHECKPOINT)
    srv.wait(rid)
    img = srv.take_image(rid)
    exp, *_ = c.oracle.checkpoint([c.host()])
    assert img.to_bytes() == exp
    img.release()
    with pytest.raises(crum.CrumError):
        srv.take_image(rid)
    rr = srv.submit(c.cid, crum.REQ_RESTORE)
    srv.wait(rr)
    with pytest.raises(crum.CrumError):
        srv.take_image(rr)
    rid2 = srv.submit(c.cid, crum.REQ_CHECKPOINT)
    srv.wait(rid2)
    srv.destroy()  # drops the image nobody took
    c.set.destroy()
    srv0 = crum.Server(staging_budget=1 << 28, max_inflight=2)
    c0 = MixClient(srv0, 1, 2 * P)
    r0 = srv0.submit(c0.cid, crum.REQ_CHECKPOINT)
    srv0.wait(r0)
    with pytest.raises(crum.CrumError):
        srv0.take_image(r0)
    srv0.destroy()
    c0.set.destroy()


def test_serving_configuration_clients_images_equal_the_oracle():
    """The serving configuration's own 32 clients (footprints log-uniform
    1 MiB..4 GiB for its seed: 11.1 GiB in all, the largest 2.7 GiB;
    int32/fp32/fp64 in turn) through a server with size-first admission and
    a 16 GiB staging budget: four rounds of the configuration's request mix
    (U[1 %, 50 %] rewrites, 80 % checkpoints with every fourth of a client
    full, 20 % restores), every checkpoint image equal to the oracle's byte
    for byte and every restore exact."""
    t = torch()
    free, _ = t.cuda.mem_get_info()
    sizes = W.workload("serving").sizes
    if free < sum(sizes) + (20 << 30):
        pytest.skip("needs about 32 GB of free device memory")
    rounds = 4
    plan = mix_plan(sizes, rounds)
    srv = crum.Server(staging_budget=16 << 30, max_inflight=8, max_checkpoints=2, max_restores=1,
                      serialize_drains=-1, keep_images=1, order=1)
    clients = [MixClient(srv, i, s) for i, s in enumerate(sizes)]
    got = run_mix(srv, clients, rounds, plan)
    stats = srv.drain()
    assert stats["failed"] == 0 and stats["completed"] == rounds * len(sizes)
    assert all(len(v) == sum(not r for r, _ in plan[i]) for i, v in got.items())
    srv.destroy()
    for c in clients:
        c.set.destroy()


def test_size_first_does_not_starve_a_large_request():
    """Size-first admission when the large client fits the staging budget
    only with no small request on the device.  Small client 7's first
    request is held on the device by a spin kernel on its stream; small
    clients 0-6 each queue a run of checkpoints behind the large request.
    The large request has waited longer than its transfer would take, so it
    holds the next free staging memory: clients 0-6 stop after a request or
    two, the large request runs as soon as client 7's request ends, and most
    of their queued requests complete after it.  (With smaller requests
    allowed to pass it, clients 0-6 run their whole queues first.)  Its image
    equals the oracle's."""
    import time
    t = torch()
    Q = 100
    budget = (64 + 4) * P
    srv = crum.Server(staging_budget=budget, max_inflight=8, max_checkpoints=-1, max_restores=-1,
                      serialize_drains=-1, order=1, keep_images=1)
    big = MixClient(srv, 0, 64 * P)
    small = [MixClient(srv, 1 + i, 8 * P) for i in range(8)]
    for c in [big] + small:  # every client's first checkpoint is full
        srv.wait(srv.submit(c.cid, crum.REQ_CHECKPOINT_FULL))
        c.oracle.checkpoint([c.host()], full=True)
    for c in [big] + small:
        c.rewrite(5, 0.5)
        c.stream.synchronize()
    with t.cuda.stream(small[7].stream):
        t.cuda._sleep(200_000_000)  # about 0.1 s at the maximum SM clock
    subs = []  # (client, request id, host time of the submit)
    for c in small:
        subs.append((c, srv.submit(c.cid, crum.REQ_CHECKPOINT), time.perf_counter()))
    t_big = time.perf_counter()
    rid = srv.submit(big.cid, crum.REQ_CHECKPOINT)
    for _ in range(Q - 1):
        for c in small[:7]:
            subs.append((c, srv.submit(c.cid, crum.REQ_CHECKPOINT), time.perf_counter()))
    info = srv.wait(rid)
    exp, *_ = big.oracle.checkpoint([big.host()])
    img = srv.take_image(rid)
    assert info["status"] == crum.OK and img.to_bytes() == exp
    img.release()
    done_big = t_big + info["t_total_ms"] / 1e3
    after = 0
    for c, r, ts in subs:
        si = srv.wait(r)
        assert si["status"] == crum.OK
        after += c is not small[7] and ts + si["t_total_ms"] / 1e3 > done_big
    srv.drain()
    srv.destroy()
    # the large request waited for client 7's held request, not for the queues
    assert info["t_queue_ms"] > 20, info
    assert after >= 7 * Q // 2, f"{after} of {7 * Q} queued small requests completed after the large one"
    for c in [big] + small:
        c.set.destroy()


def test_failed_requests_are_reported_and_the_server_continues(tmp_path):
    """Host-made failures under the server: a restore request before the
    client's first checkpoint (refused when it starts) and checkpoints whose
    file sink cannot be written (EIO once drained).  Each is reported with
    its status, counted as failed and has no image to take; the budget and
    both clients stay usable: the first client's next checkpoint equals the
    oracle's, and the sink client's next checkpoint after a failed one is
    full, as a set's is after a failed persist."""
    t = torch()
    srv = crum.Server(staging_budget=1 << 28, max_inflight=4, keep_images=1)
    a = MixClient(srv, 0, 3 * P + 4096)
    size_b = 4 * P + 8
    buf_b = t.empty(size_b, dtype=t.uint8, device="cuda")
    W.fill_(buf_b, 6200, "fp32")
    t.cuda.synchronize()
    set_b = crum.CheckpointSet(external_staging=1, sink=crum.SINK_FILE,
                               sink_dir=str(tmp_path / "missing" / "dir"))
    set_b.register(buf_b.data_ptr(), size_b)
    stream_b = t.cuda.Stream()
    cid_b = srv.add_client(set_b, stream_b.cuda_stream)

    r_restore = srv.submit(a.cid, crum.REQ_RESTORE)
    assert srv.wait(r_restore, allow=(crum.EINVAL,))["status"] == crum.EINVAL
    r_b = srv.submit(cid_b, crum.REQ_CHECKPOINT)
    info = srv.wait(r_b, allow=(crum.EIO,))
    assert info["status"] == crum.EIO and info["n_dirty"] == W.pages_of(size_b)
    for rid in (r_restore, r_b):
        with pytest.raises(crum.CrumError):
            srv.take_image(rid)

    ra = srv.submit(a.cid, crum.REQ_CHECKPOINT)
    assert srv.wait(ra)["status"] == crum.OK
    img = srv.take_image(ra)
    exp, *_ = a.oracle.checkpoint([a.host()])
    assert img.to_bytes() == exp
    img.release()
    with t.cuda.stream(stream_b):
        W.mutate_pages_(buf_b, [1], 6201)
    r_b2 = srv.submit(cid_b, crum.REQ_CHECKPOINT)
    info = srv.wait(r_b2, allow=(crum.EIO,))
    # one page rewritten, but the last image was not persisted: full again
    assert info["status"] == crum.EIO and info["n_dirty"] == W.pages_of(size_b)
    stats = srv.drain()
    assert stats["failed"] == 3 and stats["completed"] == 1
    srv.destroy()
    a.set.destroy()
    set_b.destroy()
