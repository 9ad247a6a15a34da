"""Parity at full workload sizes, in the launch configuration bench.py times
(staging halves that hold every page, autotuned mappings).  The oracle is
too slow for whole images here, so each image is checked part by part, in
full: the page table against the workload's known dirty set, every payload
slot against the pages' bytes copied from the device (valid bytes, then
zeros), every committed page hash against the oracle (hashed on all host
cores over page-aligned slices: page hashes are page-local), and the image
trailer by the oracle's image checker; a restore of the chain end onto
scribbled memory must give back the whole footprint.  At 140 GiB the page
tables and every committed hash are checked in full, payloads and the
restore on samples (a 140 GiB full image does not fit in host memory)."""
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


def make_bench_set(bufs, **cfg):
    n_pages = sum(W.pages_of(b.numel()) for b in bufs)
    s = crum.CheckpointSet(staging_bytes=2 * (n_pages + 1) * P, **cfg)
    for b in bufs:
        s.register(b.data_ptr(), b.numel())
    return s


def image_array(img, out=None):
    """The image's bytes in a (reused) host array, one copy out of the
    library's pinned buffer."""
    n = img.info()["image_bytes"]
    if out is None or out.size < n:
        out = np.empty(n, dtype=np.uint8)
    img.copy_into(out.ctypes.data, n)
    return out[:n]


def check_payload_full(img, bufs):
    """Every payload slot of an image equals its page's valid bytes, followed
    by zeros; the pages are read straight from the device allocations
    `bufs` (torch indexing, not the library) and compared on the device."""
    t = torch()
    h = parse_header(img)
    pt = page_table(img)
    n = h["n"]
    if n == 0:
        return
    payload = t.from_numpy(img[h["poff"]:h["poff"] + n * P]).to("cuda").view(n, P)
    for a in np.unique(pt[:, 0]):
        rows = np.flatnonzero(pt[:, 0] == a)
        pages = pt[rows, 1].astype(np.int64)
        buf = bufs[int(a)]
        n_full = buf.numel() // P
        full = pages < n_full
        if full.any():
            exp = buf[:n_full * P].view(n_full, P)[t.as_tensor(pages[full], device="cuda")]
            got = payload[t.as_tensor(rows[full], device="cuda")]
            assert t.equal(got, exp), f"allocation {a}"
        for r in rows[~full]:
            v = buf.numel() - n_full * P
            assert t.equal(payload[int(r), :v], buf[n_full * P:]), f"allocation {a} tail"
            assert not payload[int(r), v:].any(), f"allocation {a} tail padding"
    del payload


def test_uint32_8g_full_size():
    """The 8 GiB uint32 configuration: a full checkpoint, then 10 incremental
    checkpoints of 5 % clustered page runs, each image checked in full, then
    the chain end (full + 10 incrementals) restored onto scribbled memory
    and the whole footprint compared."""
    t = torch()
    wl = W.workload("uint32_8g")
    buf = t.empty(wl.sizes[0], dtype=t.uint8, device="cuda")
    W.fill_(buf, wl.seed, wl.kind)
    s = make_bench_set([buf])
    chain = [s.checkpoint(stream_handle(), crum.FULL)]
    chain[0].wait()
    s.autotune()
    for step in range(1, 11):
        pages = W.choose_step(wl, step, wl.n_pages)
        W.mutate_pages_(buf, pages, wl.seed + step)
        img = s.checkpoint(stream_handle())
        img.wait()
        chain.append(img)
        b = image_array(img)
        assert page_table(b)[:, 1].tolist() == pages.tolist()  # in full, ascending
        assert oracle.check_image(b) == oracle.OK               # trailer over every byte
        check_payload_full(b, [buf])
        assert np.array_equal(s.hashes(), oracle_hashes([buf.cpu().numpy()]))
        del b
    expect = buf.clone()
    W.fill_(buf, 4242, "u32")
    s.restore(chain[-1], stream_handle())
    t.cuda.synchronize()
    assert t.equal(buf, expect)
    for img in chain:
        img.release()
    s.destroy()
    del expect


def test_compressed_fp32_8g_full_size():
    """Compressed images of the 8 GiB workload with fp32 data (the kind that
    shrinks): a full checkpoint, then two incrementals of 5 % clustered
    runs.  Each incremental image in full: trailer by the oracle's checker,
    page table against the known dirty set, every slot's code equal to the
    oracle's code of that page (on all host cores), every committed hash
    against the oracle; then the chain end restored onto scribbled memory
    and the whole 8 GiB compared."""
    t = torch()
    wl = W.workload("uint32_8g")
    buf = t.empty(wl.sizes[0], dtype=t.uint8, device="cuda")
    W.fill_(buf, wl.seed + 5, "fp32")
    s = make_bench_set([buf], compress=1)
    chain = [s.checkpoint(stream_handle(), crum.FULL)]
    chain[0].wait()
    n_full = wl.n_pages
    for step in (1, 2):
        pages = W.choose_step(wl, 100 + step, n_full)
        W.mutate_pages_(buf, pages, wl.seed + 100 + step)
        img = s.checkpoint(stream_handle())
        img.wait()
        chain.append(img)
        b = image_array(img)
        h = parse_header(b)
        n, A = h["n"], h["A"]
        assert oracle.image_version(b) == 2 and oracle.check_image(b) == oracle.OK
        assert page_table(b)[:, 1].tolist() == pages.tolist()
        offs = np.frombuffer(b, dtype=np.uint64, count=n, offset=64 + 16 * A + 16 * n).astype(np.int64)
        ends = np.append(offs[1:], h["size"] - 8 - h["poff"])
        host = buf.cpu().numpy().reshape(n_full, P)

        def slot_ok(j):
            code = b[h["poff"] + offs[j]:h["poff"] + ends[j]].tobytes()
            return code == oracle.bpd_encode(host[pages[j]])

        with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
            ok = list(ex.map(slot_ok, range(n)))
        assert all(ok), f"step {step}: {ok.count(False)} slots differ from the oracle's code"
        assert np.array_equal(s.hashes(), oracle_hashes([host.reshape(-1)]))
        del b, host
    expect = buf.clone()
    W.fill_(buf, 4243, "u32")
    s.restore(chain[-1], stream_handle())
    t.cuda.synchronize()
    assert t.equal(buf, expect)
    for img in chain:
        img.release()
    s.destroy()
    del expect


def test_stencil_full_size():
    """The stencil configuration (200 fp64 fields, 24 GiB): 20 checkpoints,
    each after a 27-point stencil step over interior z-ranges (30 % of
    pages), batched, autotuned; every image checked in full (page table,
    payload, trailer of the first and last; committed hashes against the
    oracle at the first new chain and at the end), then the chain end restored onto scribbled memory and
    the whole footprint compared.  A chain is capped at 5 incrementals
    (``max_chain``) so that host memory holds one chain (24 GiB + 5 x 7 GiB):
    checkpoints 6, 12 and 18 are full, and the chain end (checkpoint 20) is
    the full image of checkpoint 18 plus two incrementals."""
    t = torch()
    wl = W.workload("stencil")
    bufs = []
    for i, n in enumerate(wl.sizes):
        b = t.empty(n, dtype=t.uint8, device="cuda")
        W.fill_(b, wl.seed * 7919 + i, wl.kind)
        bufs.append(b)
    s = make_bench_set(bufs, max_chain=5)
    s.checkpoint(stream_handle(), crum.FULL).wait()
    s.autotune()
    plane = 8 * W.STENCIL_NX * W.STENCIL_NY
    last, arr = None, None
    for step in range(1, 21):
        plans = [W.stencil_plan(n, wl.dirty_frac, 77 + 1000 * step + i) for i, n in enumerate(wl.sizes)]
        for b, plan in zip(bufs, plans):
            W.stencil_step_(b, plan)
        img = s.checkpoint(stream_handle())
        img.wait()
        arr = image_array(img, arr)
        b = arr[:img.info()["image_bytes"]]
        hdr = parse_header(b)
        if hdr["flags"] & 1:  # every sixth image starts a new chain
            assert step % 6 == 0 and hdr["n"] == wl.n_pages
        else:
            exp = []
            for a, plan in enumerate(plans):
                if plan is not None:
                    _, z0, L = plan
                    exp.extend((a, p) for p in range(z0 * plane // P, ((z0 + L) * plane - 1) // P + 1))
            assert page_table(b).tolist() == [list(x) for x in exp]  # in full
        assert (hdr["flags"] & 1) == (step % 6 == 0)
        if step in (1, 20):
            assert oracle.check_image(b) == oracle.OK
        check_payload_full(b, bufs)
        if step in (6, 20):
            assert np.array_equal(s.hashes(), oracle_hashes([x.cpu().numpy() for x in bufs]))
        del b
        if last is not None:
            last.release()
        last = img
    expect = [x.clone() for x in bufs]
    for i, x in enumerate(bufs):
        W.fill_(x, 555 + i, "u32")
    s.restore(last, stream_handle())
    t.cuda.synchronize()
    assert all(t.equal(x, e) for x, e in zip(bufs, expect))
    last.release()
    s.destroy()
    del expect


def test_large_4096_allocations_sampled():
    """The 140 GiB / 4,096-allocation footprint: the base image is drained
    without keeping its payload (it exceeds host memory); two incremental
    steps of a seeded 2 % scatter are checked: page table in full, the image
    checksum by the oracle's checker, every payload slot against the pages
    gathered on the device in 4 KiB blocks (allocation sizes are 4 KiB
    multiples), committed hashes on a seeded sample of pages after each
    step, and after the last step every committed hash (2.3 million pages)
    against the oracle's, 8 GiB of the footprint at a time on all host
    cores."""
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
    sizes_np = np.asarray(wl.sizes, dtype=np.int64)
    assert not (sizes_np % 4096).any()
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
        b = image_array(img)
        pt = page_table(b)
        assert pt[:, 0].tolist() == page_alloc[chosen].tolist()
        assert pt[:, 1].tolist() == page_local[chosen].tolist()
        assert oracle.check_image(b) == oracle.OK
        h = parse_header(b)
        hashes = s.hashes()
        n = h["n"]
        valid = np.minimum(P, sizes_np[page_alloc[chosen]] - page_local[chosen] * P)
        cnt = valid // 4096
        within = np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        src_blk = np.repeat((offs[page_alloc[chosen]] + page_local[chosen] * P) // 4096, cnt) + within
        dst_blk = np.repeat(np.arange(n) * (P // 4096), cnt) + within
        exp = t.zeros((n * (P // 4096), 4096), dtype=t.uint8, device="cuda")
        exp[t.as_tensor(dst_blk, device="cuda")] = big.view(-1, 4096)[t.as_tensor(src_blk, device="cuda")]
        payload = np.frombuffer(b, dtype=np.uint8, count=n * P, offset=h["poff"])
        assert np.array_equal(exp.cpu().numpy().reshape(-1), payload)
        del exp
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
