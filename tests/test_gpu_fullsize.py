"""Parity at full workload sizes, in the launch configuration bench.py times
(staging halves that hold every page, autotuned mappings).  The oracle is
too slow for whole images here, so: page tables are checked in full against
the workload's known dirty set, every page hash against the oracle (hashed
on all host cores over page-aligned slices: page hashes are page-local),
the incremental image's checksum by the oracle's image checker, payload
slots on a seeded sample, and the restored chain on a seeded sample."""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import pytest

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W

from helpers import page_table, parse_header, stream_handle, torch

pytestmark = pytest.mark.gpu
P = 65536


@pytest.fixture(autouse=True)
def _cuda():
    t = torch()
    if not t.cuda.is_available():
        pytest.skip("needs a CUDA device")
    free, _ = t.cuda.mem_get_info()
    if free < 100 << 30:
        pytest.skip("needs about 100 GB of free device memory")
    crum.load()
    yield
    t.cuda.synchronize()
    t.cuda.empty_cache()


def oracle_hashes(host_allocs, chunk_pages=4096):
    """Oracle page hashes of every page, in global page order, computed in
    parallel over page-aligned slices (the C oracle releases the GIL)."""
    jobs = []
    for a in host_allocs:
        for lo in range(0, a.size, chunk_pages * P):
            jobs.append(a[lo:lo + chunk_pages * P])
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        parts = list(ex.map(lambda x: oracle.hash_all([x]), jobs))
    return np.concatenate(parts)


def make_bench_set(bufs):
    n_pages = sum(W.pages_of(b.numel()) for b in bufs)
    s = crum.CheckpointSet(staging_bytes=2 * (n_pages + 1) * P)
    for b in bufs:
        s.register(b.data_ptr(), b.numel())
    return s


def check_image_sample(img_bytes, host_allocs, offsets, rng, n_sample=64):
    h = parse_header(img_bytes)
    pt = page_table(img_bytes)
    idx = rng.choice(h["n"], size=min(n_sample, h["n"]), replace=False)
    for s in idx:
        a, p = int(pt[s, 0]), int(pt[s, 1])
        src = host_allocs[a][p * P:(p + 1) * P]
        slot = np.frombuffer(img_bytes, dtype=np.uint8, count=P, offset=h["poff"] + int(s) * P)
        assert np.array_equal(slot[:src.size], src) and not slot[src.size:].any(), f"slot {s}"


def test_uint32_8g_full_size():
    t = torch()
    wl = W.workload("uint32_8g")
    buf = t.empty(wl.sizes[0], dtype=t.uint8, device="cuda")
    W.fill_(buf, wl.seed, wl.kind)
    s = make_bench_set([buf])
    s.checkpoint(stream_handle(), crum.FULL).wait()
    s.autotune()
    chain, rng = [], np.random.default_rng(11)
    for step in (1, 2):
        pages = W.choose_step(wl, step, wl.n_pages)
        W.mutate_pages_(buf, pages, wl.seed + step)
        img = s.checkpoint(stream_handle())
        img.wait()
        chain.append(img)
        b = img.to_bytes()
        assert page_table(b)[:, 1].tolist() == pages.tolist()  # in full, ascending
        assert oracle.check_image(b) == oracle.OK               # trailer over every byte
        host = buf.cpu().numpy()
        check_image_sample(b, [host], [0], rng)
        assert np.array_equal(s.hashes(), oracle_hashes([host]))
        del b
    state = buf.cpu().numpy()
    sample = rng.choice(wl.n_pages, size=256, replace=False)
    W.fill_(buf, 4242, "u32")
    s.restore(chain[-1], stream_handle())
    t.cuda.synchronize()
    got = buf.cpu().numpy()
    for p in sample:
        assert np.array_equal(got[p * P:(p + 1) * P], state[p * P:(p + 1) * P]), p
    for img in chain:
        img.release()
    s.destroy()


def test_stencil_full_size():
    t = torch()
    wl = W.workload("stencil")
    bufs = []
    for i, n in enumerate(wl.sizes):
        b = t.empty(n, dtype=t.uint8, device="cuda")
        W.fill_(b, wl.seed * 7919 + i, wl.kind)
        bufs.append(b)
    s = make_bench_set(bufs)
    s.checkpoint(stream_handle(), crum.FULL).wait()
    s.autotune()
    offsets = np.cumsum([0] + [W.pages_of(n) for n in wl.sizes])
    plans = [W.stencil_plan(n, wl.dirty_frac, 77 + i) for i, n in enumerate(wl.sizes)]
    for b, plan in zip(bufs, plans):
        W.stencil_step_(b, plan)
    img = s.checkpoint(stream_handle())
    img.wait()
    b = img.to_bytes()
    plane = 8 * W.STENCIL_NX * W.STENCIL_NY
    exp = []
    for a, plan in enumerate(plans):
        if plan is not None:
            _, z0, L = plan
            exp.extend((a, p) for p in range(z0 * plane // P, ((z0 + L) * plane - 1) // P + 1))
    assert page_table(b).tolist() == [list(x) for x in exp]  # in full
    assert oracle.check_image(b) == oracle.OK
    hosts = [x.cpu().numpy() for x in bufs]
    check_image_sample(b, hosts, offsets, np.random.default_rng(5))
    assert np.array_equal(s.hashes(), oracle_hashes(hosts))
    img.release()
    s.destroy()


def test_large_4096_allocations_sampled():
    """The 140 GiB / 4,096-allocation footprint: the base image is drained
    without keeping its payload (it exceeds host memory); two incremental
    steps of a seeded 2 % scatter are checked: page table in full, the image
    checksum by the oracle's checker, sampled payload slots, committed hashes
    on a seeded sample of pages after each step, and after the last step
    every committed hash (2.3 million pages) against the oracle's, 8 GiB of
    the footprint at a time on all host cores."""
    t = torch()
    free, _ = t.cuda.mem_get_info()
    wl = W.workload("large")
    if free < wl.total_bytes + (24 << 30):
        pytest.skip("needs about 165 GB of free device memory")
    S = wl.total_bytes
    big = W.managed_empty(S)  # the configuration names device-resident managed memory
    W.fill_(big, wl.seed, wl.kind)
    offs = np.cumsum([0] + list(wl.sizes))
    bufs = [big[int(offs[i]):int(offs[i + 1])] for i in range(len(wl.sizes))]
    first = np.cumsum([0] + [W.pages_of(n) for n in wl.sizes])
    page_alloc = np.repeat(np.arange(len(wl.sizes)), np.diff(first))
    page_local = np.arange(wl.n_pages) - first[page_alloc]
    k = int(round(wl.dirty_frac * wl.n_pages))
    s = crum.CheckpointSet(staging_bytes=2 * (int(1.5 * k) + 1) * P)
    for b in bufs:
        s.register(b.data_ptr(), b.numel())
    s.checkpoint(stream_handle(), crum.FULL | crum.NO_PAYLOAD).wait()
    big64 = big.view(t.int64)
    rng = np.random.default_rng(3)
    for step in (1, 2):
        chosen = W.choose_step(wl, step, wl.n_pages)
        words = (offs[page_alloc[chosen]] + page_local[chosen] * P) // 8
        idx = t.as_tensor(words, device="cuda")
        big64[idx] = big64[idx] ^ t.as_tensor(rng.integers(1, 2**62, size=chosen.size) | 1,
                                              device="cuda")
        img = s.checkpoint(stream_handle())
        img.wait()
        b = img.to_bytes()
        pt = page_table(b)
        assert pt[:, 0].tolist() == page_alloc[chosen].tolist()
        assert pt[:, 1].tolist() == page_local[chosen].tolist()
        assert oracle.check_image(b) == oracle.OK
        h = parse_header(b)
        hashes = s.hashes()
        for slot in rng.choice(h["n"], size=64, replace=False):
            a, p = int(pt[slot, 0]), int(pt[slot, 1])
            lo = int(offs[a]) + p * P
            n_valid = min(P, int(wl.sizes[a]) - p * P)
            page = big[lo:lo + n_valid].cpu().numpy()
            got = np.frombuffer(b, dtype=np.uint8, count=P, offset=h["poff"] + int(slot) * P)
            assert np.array_equal(got[:n_valid], page)
        for g in rng.choice(wl.n_pages, size=512, replace=False):
            a = int(page_alloc[g])
            lo = int(offs[a]) + int(page_local[g]) * P
            n_valid = min(P, int(wl.sizes[a]) - int(page_local[g]) * P)
            assert int(hashes[g]) == oracle.page_hash(big[lo:lo + n_valid].cpu().numpy())
        img.release()
    hashes = s.hashes()
    g0, group, acc = 0, [], 0
    for a in range(len(wl.sizes)):
        group.append(a)
        acc += int(wl.sizes[a])
        if acc >= (8 << 30) or a == len(wl.sizes) - 1:
            host = [big[int(offs[k]):int(offs[k + 1])].cpu().numpy() for k in group]
            exp = oracle_hashes(host)
            assert np.array_equal(hashes[g0:g0 + exp.size], exp), f"allocations {group[0]}-{group[-1]}"
            g0 += exp.size
            group, acc = [], 0
            del host
    assert g0 == wl.n_pages
    s.destroy()
    del big


@pytest.mark.parametrize("mode", [crum.RESTORE_MERGED, crum.RESTORE_REPLAY])
def test_large_shape_restore_from_the_chain(mode):
    """The large configuration's shape (4,096 managed allocations, sizes
    log-uniform 64 KiB-2 GiB) at 40 GiB, the most the host can hold as a kept
    full image: a full image and two incrementals of a 2 % scatter, the
    memory scribbled, the chain end restored; the whole footprint must equal
    its state at the chain end (compared on the device byte for byte) and
    sampled pages equal the host copies taken before the scribble."""
    t = torch()
    sizes = W.loguniform_sizes(0x5EED + 4, 4096, 64 << 10, 2 << 30, 40 << 30)
    S = sum(sizes)
    free, _ = t.cuda.mem_get_info()
    if free < 2 * S + (16 << 30):
        pytest.skip("needs about 100 GB of free device memory")
    big = W.managed_empty(S)
    W.fill_(big, 0x5EED + 4, "fp32")
    offs = np.cumsum([0] + list(sizes))
    bufs = [big[int(offs[i]):int(offs[i + 1])] for i in range(len(sizes))]
    n_pages = sum(W.pages_of(n) for n in sizes)
    first = np.cumsum([0] + [W.pages_of(n) for n in sizes])
    page_alloc = np.repeat(np.arange(len(sizes)), np.diff(first))
    page_local = np.arange(n_pages) - first[page_alloc]
    k = int(round(0.02 * n_pages))
    s = crum.CheckpointSet(staging_bytes=2 * (int(1.5 * k) + 1) * P, restore_mode=mode)
    for b in bufs:
        s.register(b.data_ptr(), b.numel())
    chain = [s.checkpoint(stream_handle(), crum.FULL)]
    chain[0].wait()
    big64 = big.view(t.int64)
    rng = np.random.default_rng(41)
    for step in (1, 2):
        chosen = np.sort(rng.choice(n_pages, size=k, replace=False))
        words = t.as_tensor((offs[page_alloc[chosen]] + page_local[chosen] * P) // 8, device="cuda")
        big64[words] = big64[words] ^ t.as_tensor(rng.integers(1, 2**62, size=k) | 1, device="cuda")
        img = s.checkpoint(stream_handle())
        img.wait()
        chain.append(img)
    t.cuda.synchronize()
    expect = big.clone()
    sample = rng.choice(n_pages, size=256, replace=False)
    def page_bytes(g):
        a = int(page_alloc[g])
        lo = int(offs[a]) + int(page_local[g]) * P
        return big[lo:lo + min(P, int(sizes[a]) - int(page_local[g]) * P)].cpu().numpy()
    before = [page_bytes(g) for g in sample]
    W.fill_(big, 77, "u32")
    s.restore(chain[-1], stream_handle())
    t.cuda.synchronize()
    assert t.equal(big, expect)
    assert all(np.array_equal(page_bytes(g), b) for g, b in zip(sample, before))
    for c in chain:
        c.release()
    s.destroy()
    del big, expect
