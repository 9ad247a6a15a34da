"""Seeded random scenarios through the C ABI against the oracle: random
allocation sizes (tiny, ragged, several pages), staging that holds every
page or only a few (chunked capture), graph or plain launches, random hash
and gather mappings, verify sets, compressed images (chunked too), four
data kinds, managed memory whose pages the scenario places on the device or
the host (read in place or migrated), drain copy sizes down to 4 KiB, and
per step a random rewrite and a random checkpoint flag (incremental, full,
verify, no payload); now and then the
chain end is restored onto scribbled memory with the scenario's restore
form.  Every image is compared with the oracle's byte for byte (checksum
and size when the payload is not kept)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W

from helpers import device_buffers, first_diff, host_copies, make_set, stream_handle, torch

pytestmark = pytest.mark.gpu
P = W.PAGE


@pytest.fixture(autouse=True)
def _cuda():
    t = torch()
    if not t.cuda.is_available():
        pytest.skip("needs a CUDA device")
    crum.load()
    yield
    t.cuda.synchronize()


def _sizes(rng):
    out = []
    for _ in range(int(rng.integers(1, 7))):
        kind = rng.integers(0, 4)
        if kind == 0:
            out.append(int(rng.integers(1, 200)))
        elif kind == 1:
            out.append(int(rng.integers(1, P)))
        elif kind == 2:
            out.append(int(rng.integers(1, 6)) * P)
        else:
            out.append(int(rng.integers(2, 40)) * P + int(rng.integers(1, P)))
    return out


def _rewrite(bufs, sizes, frac, rng):
    for b, n in zip(bufs, sizes):
        pages = W.pages_of(n)
        k = int(round(frac * pages))
        if k:
            W.mutate_pages_(b, np.sort(rng.choice(pages, size=k, replace=False)),
                            int(rng.integers(1, 1 << 30)))
    torch().cuda.synchronize()


@pytest.mark.parametrize("seed", range(64))
def test_random_scenario(seed):
    rng = np.random.default_rng(1000 + seed)
    sizes = _sizes(rng)
    n_pages = sum(W.pages_of(n) for n in sizes)
    chunked = bool(rng.integers(0, 2))
    verify = bool(rng.integers(0, 2))
    compress = bool(rng.integers(0, 2))
    managed = int(rng.integers(0, 3)) == 0
    in_place = managed and bool(rng.integers(0, 2))
    cfg = dict(staging_bytes=(2 * int(rng.integers(1, 4)) * P) if chunked else 2 * (n_pages + 1) * P,
               use_graph=int(rng.integers(0, 2)), hash_mapping=int(rng.integers(0, crum.NUM_HASH_MAPPINGS)),
               gather_mapping=int(rng.integers(0, 6)), verify=int(verify),
               restore_mode=int(rng.integers(0, 4)), compress=int(compress),
               managed_in_place=int(in_place),
               chunk_bytes=int(rng.choice([0, 4096, 12304, 1 << 20])))
    kind = ["u32", "fp32", "fp64", "bf16"][seed % 4]
    if managed:
        bufs = []
        for i, n in enumerate(sizes):
            b = W.managed_empty(n)
            W.fill_(b, (seed + 50) * 7919 + i, kind)
            bufs.append(b)
        torch().cuda.synchronize()
        for b in bufs:
            if rng.integers(0, 2):
                W.managed_prefetch(b.data_ptr(), b.numel(), "host")
    else:
        bufs = device_buffers(sizes, seed=seed + 50, kind=kind)
    s = make_set(bufs, **cfg)
    o = oracle.OracleSet(sizes, compress=compress)
    chain_ok = False  # every image since the last full one kept its payload
    chain_end, state_end = None, None
    images = []
    force_full = False
    for step in range(7):
        if step:
            _rewrite(bufs, sizes, float(rng.choice([0.0, 0.1, 0.5, 1.0])), rng)
        choice = int(rng.integers(0, 10))
        flags = crum.INCR
        if choice == 0:
            flags = crum.FULL
        elif choice == 1:
            flags = crum.NO_PAYLOAD
        elif choice in (2, 3) and verify:
            flags = crum.VERIFY
        full = step == 0 or flags == crum.FULL or force_full
        force_full = False
        img = s.checkpoint(stream_handle(), flags)
        img.wait()
        state = host_copies(bufs)
        exp, *_ = o.checkpoint(state, full=full)
        info = img.info()
        assert info["full"] == int(full), (step, cfg)
        assert info["checksum"] == int(np.frombuffer(exp[-8:], dtype=np.uint64)[0]), (step, cfg)
        assert info["image_bytes"] == len(exp)
        if flags == crum.NO_PAYLOAD:
            chain_ok = False
        else:
            assert first_diff(img.to_bytes(), exp) is None, (step, cfg)
            chain_ok = chain_ok or full
            if full:
                chain_ok = True
        images.append(img)
        chain_end, state_end = img, state
        if step in (3, 6) and chain_ok:
            # scribble a third of the pages, then restore the chain end
            _rewrite(bufs, sizes, 0.34, rng)
            s.restore(chain_end, stream_handle())
            torch().cuda.synchronize()
            got = host_copies(bufs)
            assert all(np.array_equal(g, w) for g, w in zip(got, state_end)), (step, cfg)
            force_full = verify  # the verify shadow does not hold restored bytes
    for im in images:
        im.release()
    s.destroy()


def test_sets_used_from_several_host_threads():
    """Four host threads, each with its own set, stream and allocations,
    checkpoint and restore at the same time; every image matches the
    oracle's and every restore returns its thread's memory."""
    import threading
    t = torch()
    errors = []

    def worker(k):
        try:
            rng = np.random.default_rng(500 + k)
            sizes = [int(rng.integers(1, 20)) * P + int(rng.integers(0, P)), 3 * P]
            stream = t.cuda.Stream()
            with t.cuda.stream(stream):
                bufs = [t.empty(n, dtype=t.uint8, device="cuda") for n in sizes]
                for i, b in enumerate(bufs):
                    W.fill_(b, 900 + 10 * k + i, "u32")
            stream.synchronize()
            s = crum.CheckpointSet(restore_mode=int(k % 4))
            for b in bufs:
                s.register(b.data_ptr(), b.numel())
            o = oracle.OracleSet(sizes)
            imgs = []
            for step in range(5):
                if step:
                    with t.cuda.stream(stream):
                        for i, (b, n) in enumerate(zip(bufs, sizes)):
                            pages = W.pages_of(n)
                            W.mutate_pages_(b, np.sort(rng.choice(pages, size=max(1, pages // 3), replace=False)),
                                            100 * k + 10 * step + i)
                img = s.checkpoint(stream.cuda_stream)
                img.wait()
                stream.synchronize()
                state = [b.cpu().numpy().copy() for b in bufs]
                exp, *_ = o.checkpoint(state)
                if first_diff(img.to_bytes(), exp) is not None:
                    errors.append(f"thread {k} step {step}: image differs")
                imgs.append(img)
            with t.cuda.stream(stream):
                for b in bufs:
                    b.fill_(0xAB)
            s.restore(imgs[-1], stream.cuda_stream)
            stream.synchronize()
            if not all(np.array_equal(b.cpu().numpy(), w) for b, w in zip(bufs, state)):
                errors.append(f"thread {k}: restore differs")
            for im in imgs:
                im.release()
            s.destroy()
        except Exception as e:  # reported below, on the main thread
            errors.append(f"thread {k}: {e!r}")

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
