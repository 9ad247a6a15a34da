"""Managed (unified) memory, the paper's subject: allocations made with
cudaMallocManaged are registered like device memory and must give the same
bit-exact images and restores, whether their pages sit on the device or on
the host when the checkpoint runs; with managed_in_place, host-placed pages
are read where they are and stay there.  Registration rejects memory the
kernels cannot read."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W

from helpers import first_diff, host_copies, make_set, stream_handle, torch

pytestmark = pytest.mark.gpu
P = W.PAGE
SIZES = [1, 24, P - 8, P, 3 * P + 40, 37 * P + 4104]


@pytest.fixture(autouse=True)
def _cuda():
    t = torch()
    if not t.cuda.is_available():
        pytest.skip("needs a CUDA device")
    crum.load()
    yield
    t.cuda.synchronize()


def _managed(sizes, seed):
    bufs = []
    for i, n in enumerate(sizes):
        b = W.managed_empty(n)
        W.fill_(b, seed * 7919 + i, "u32")
        bufs.append(b)
    torch().cuda.synchronize()
    return bufs


def _ckpt(s, flags=crum.INCR):
    img = s.checkpoint(stream_handle(), flags)
    img.wait()
    return img, img.to_bytes()


def _mutate(bufs, frac, seed):
    for i, b in enumerate(bufs):
        n = W.pages_of(b.numel())
        k = max(1, int(round(frac * n)))
        W.mutate_pages_(b, W.choose_uniform(seed * 31 + i, n, k), seed * 131 + i)
    torch().cuda.synchronize()


@pytest.mark.parametrize("where", ["device", "host"])
def test_managed_chain_and_restore(where):
    """Full + two incrementals of managed allocations against the oracle;
    before each checkpoint the pages are moved to `where` (host-resident
    pages migrate back as the kernels read them); then the chain end is
    restored onto garbage through both restore forms."""
    bufs = _managed(SIZES, seed=71)
    o = oracle.OracleSet(SIZES)
    states, chain = [], []
    s = make_set(bufs)
    for step in range(3):
        if step:
            _mutate(bufs, 0.4, seed=710 + step)
        states.append(host_copies(bufs))
        for b in bufs:
            W.managed_prefetch(b.data_ptr(), b.numel(), where)
        img, got = _ckpt(s)
        exp, *_ = o.checkpoint(states[-1])
        assert first_diff(got, exp) is None, f"step {step}"
        chain.append(img)
    for mode in (crum.RESTORE_REPLAY, crum.RESTORE_MERGED):
        r = make_set(bufs, restore_mode=mode)
        for i, b in enumerate(bufs):
            W.fill_(b, 9000 + i, "u32")
        if where == "host":
            for b in bufs:
                W.managed_prefetch(b.data_ptr(), b.numel(), "host")
        r.restore(chain[-1], stream_handle())
        torch().cuda.synchronize()
        assert all(np.array_equal(g, w) for g, w in zip(host_copies(bufs), states[-1])), mode
        r.destroy()
    for c in chain:
        c.release()
    s.destroy()


def test_managed_and_device_memory_in_one_set():
    t = torch()
    sizes = [5 * P + 8, 2 * P]
    m = _managed(sizes[:1], seed=73)[0]
    d = t.empty(sizes[1], dtype=t.uint8, device="cuda")
    W.fill_(d, 74, "u32")
    s = make_set([m, d])
    img, got = _ckpt(s)
    exp, *_ = oracle.OracleSet(sizes).checkpoint(host_copies([m, d]))
    assert first_diff(got, exp) is None
    img.release()
    s.destroy()


def test_registration_rejects_memory_kernels_cannot_read():
    t = torch()
    s = crum.CheckpointSet()
    pinned = t.empty(4 * P, dtype=t.uint8).pin_memory()
    pageable = np.zeros(4 * P + 16, dtype=np.uint8)
    addr = pageable.ctypes.data + (-pageable.ctypes.data) % 16
    dev = t.empty(4 * P, dtype=t.uint8, device="cuda")
    for ptr, n in [(pinned.data_ptr(), 4 * P), (addr, 4 * P), (dev.data_ptr(), 2 * P + (1 << 40))]:
        with pytest.raises(crum.CrumError) as e:
            s.register(ptr, n)
        assert e.value.status == crum.EINVAL
    s.register(dev.data_ptr(), 4 * P)
    s.destroy()


def _read_gbs(b):
    """Rate of one device page-hash pass over b (best of three), GB/s."""
    t = torch()
    out = t.empty(W.pages_of(b.numel()), dtype=t.int64, device="cuda")
    best = 1e30
    for _ in range(3):
        e0, e1 = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
        e0.record()
        crum.hash_pages(b.data_ptr(), b.numel(), out.data_ptr(), stream_handle())
        e1.record()
        t.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return b.numel() / best / 1e6


def test_host_placed_managed_pages_are_read_in_place():
    """Section 4.4's oversubscribed case in small: one allocation on the
    device, one the application prefetched to the host, one whose preferred
    location is the host.  With managed_in_place the images and restores are
    bit-exact and the host-placed pages are still in host memory afterwards
    (a device pass over them runs at the link's rate, not HBM's); the set's
    advice is withdrawn when it is destroyed, the application's own is kept."""
    sizes = [512 * P + 40, 128 * P * 16, 8 * P * 16 + 8]
    bufs = _managed(sizes, seed=75)
    dev_buf, host_buf, pref_buf = bufs
    W.managed_advise(pref_buf.data_ptr(), pref_buf.numel(), "preferred_host")
    mine = W.managed_empty(4 * P)
    W.managed_advise(mine.data_ptr(), mine.numel(), "accessed_by")

    def place():
        # host copies go through the copy engine; put the pages back where the
        # application keeps them before each checkpoint
        for b in (host_buf, pref_buf, mine):
            W.managed_prefetch(b.data_ptr(), b.numel(), "host")

    host_pages = W.pages_of(sizes[1]) + W.pages_of(sizes[2])
    o = oracle.OracleSet(sizes)
    s = make_set(bufs, managed_in_place=1)
    probe = make_set([mine], managed_in_place=1)
    chain, states = [], []
    for step in range(3):
        if step:
            _mutate(bufs, 0.3, seed=750 + step)
        states.append(host_copies(bufs))
        place()
        img, got = _ckpt(s)
        assert img.info()["host_pages"] == host_pages
        # 128 MiB: over the link ~50 GB/s; from HBM (had it migrated) > 1 TB/s
        assert _read_gbs(host_buf) < 200, "host-placed pages migrated"
        assert _read_gbs(dev_buf) > 400
        exp, *_ = o.checkpoint(states[-1])
        assert first_diff(got, exp) is None, f"step {step}"
        chain.append(img)
    assert 0 in W.managed_accessed_by(host_buf.data_ptr(), host_buf.numel())
    assert 0 not in W.managed_accessed_by(dev_buf.data_ptr(), dev_buf.numel())
    for mode in (crum.RESTORE_REPLAY, crum.RESTORE_MERGED, crum.RESTORE_DELTA):
        r = make_set(bufs, restore_mode=mode, managed_in_place=1)
        for i, b in enumerate(bufs):
            W.fill_(b, 7500 + i, "u32")
        place()
        r.restore(chain[-1], stream_handle())
        torch().cuda.synchronize()
        assert _read_gbs(host_buf) < 200, f"restore migrated host-placed pages ({mode})"
        assert all(np.array_equal(g, w) for g, w in zip(host_copies(bufs), states[-1])), mode
        r.destroy()
    for c in chain:
        c.release()
    probe.checkpoint(stream_handle()).wait()
    s.destroy()
    probe.destroy()
    assert 0 not in W.managed_accessed_by(host_buf.data_ptr(), host_buf.numel())
    assert 0 not in W.managed_accessed_by(pref_buf.data_ptr(), pref_buf.numel())
    assert 0 in W.managed_accessed_by(mine.data_ptr(), mine.numel())


def test_managed_placement_left_alone_by_default():
    b = _managed([16 * P], seed=77)[0]
    W.managed_prefetch(b.data_ptr(), b.numel(), "host")
    s = make_set([b])
    img, got = _ckpt(s)
    assert img.info()["host_pages"] == 0
    assert 0 not in W.managed_accessed_by(b.data_ptr(), b.numel())
    exp, *_ = oracle.OracleSet([16 * P]).checkpoint(host_copies([b]))
    assert first_diff(got, exp) is None
    s.destroy()


def test_advice_follows_the_application_placement():
    """A range prefetched back to the device loses the set's advice at the
    next checkpoint, and gets it again once it is back in host memory."""
    sizes = [12 * P + 8]
    b = _managed(sizes, seed=79)[0]
    s = make_set([b], managed_in_place=1)
    o = oracle.OracleSet(sizes)
    for k, (where, advised) in enumerate((("host", True), ("device", False), ("host", True))):
        _mutate([b], 0.5, seed=790 + k)
        state = host_copies([b])
        W.managed_prefetch(b.data_ptr(), b.numel(), where)
        img, got = _ckpt(s)
        assert (0 in W.managed_accessed_by(b.data_ptr(), b.numel())) == advised, where
        assert img.info()["host_pages"] == (W.pages_of(sizes[0]) if advised else 0)
        exp, *_ = o.checkpoint(state)
        assert first_diff(got, exp) is None, where
        img.release()
    s.destroy()
    assert 0 not in W.managed_accessed_by(b.data_ptr(), b.numel())
