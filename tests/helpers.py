"""Shared plumbing of the GPU parity tests: device buffers, host copies and
oracle sets.  No method arithmetic here: hashes, dirty sets and images come
from the oracle (expected) and from the CUDA library (actual)."""
from __future__ import annotations

import numpy as np

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W


def torch():
    import torch as _t
    return _t


def device_buffers(sizes, seed, kind="u32"):
    """One uint8 CUDA tensor per size, seeded; allocations are 256-byte aligned."""
    t = torch()
    bufs = []
    for i, n in enumerate(sizes):
        b = t.empty(n, dtype=t.uint8, device="cuda")
        W.fill_(b, seed * 7919 + i, kind)
        bufs.append(b)
    t.cuda.synchronize()
    return bufs


def host_copies(bufs):
    torch().cuda.synchronize()
    return [b.cpu().numpy().copy() for b in bufs]


def make_set(bufs, **cfg):
    s = crum.CheckpointSet(**cfg)
    for b in bufs:
        s.register(b.data_ptr(), b.numel())
    return s


def stream_handle():
    return torch().cuda.current_stream().cuda_stream


def page_offsets(sizes):
    """Global page index of page 0 of each allocation."""
    out, g = [], 0
    for n in sizes:
        out.append(g)
        g += W.pages_of(n)
    return out


def mutate(bufs, sizes, frac, seed):
    """Mutate a uniform random fraction of each allocation's pages on the
    device; returns the set of global pages touched."""
    touched = set()
    for i, (b, g0) in enumerate(zip(bufs, page_offsets(sizes))):
        n = W.pages_of(sizes[i])
        k = int(round(frac * n))
        if k == 0:
            continue
        pages = W.choose_uniform(seed * 31 + i, n, k)
        W.mutate_pages_(b, pages, seed * 131 + i)
        touched.update(int(g0 + p) for p in pages)
    torch().cuda.synchronize()
    return touched


def parse_header(img: bytes):
    import struct
    magic, ver, flags, seq, parent, psz, A, n, poff, size = struct.unpack_from("<8sIIQQIIQQQ", img, 0)
    return dict(magic=magic, ver=ver, flags=flags, seq=seq, parent=parent, psz=psz, A=A, n=n,
                poff=poff, size=size)


def page_table(img: bytes):
    h = parse_header(img)
    a = np.frombuffer(img, dtype=np.uint32, count=2 * h["n"], offset=64 + 16 * h["A"])
    return a.reshape(-1, 2)


def first_diff(a: bytes, b: bytes):
    if len(a) != len(b):
        return f"length {len(a)} != {len(b)}"
    x = np.frombuffer(a, dtype=np.uint8)
    y = np.frombuffer(b, dtype=np.uint8)
    idx = np.flatnonzero(x != y)
    return None if idx.size == 0 else f"{idx.size} bytes differ, first at {idx[0]}"
