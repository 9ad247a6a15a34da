"""CPU oracle for the CRUM capture/restore path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports,
links or runs it, and it shares no code with the CUDA path.

Two independent renderings of the method live here:

* ``crum_oracle.c`` -- plain C, loaded through ctypes: page hash, dirty rule,
  verify mode, image writer/checker and restore (see the comment at its top
  for the passages of the paper each step follows).
* ``bigint`` -- a pure-Python big-integer rendering of the hash alone, for
  tiny inputs, used to cross-check the C code.

Wrappers below take and return numpy arrays and ``bytes``; they add no
arithmetic of their own.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Sequence

import numpy as np

PAGE = 65536
OK, CORRUPT, MISMATCH = 0, -1, -2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crum_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcrum_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``crum_oracle.c`` with gcc into ``oracle/_build``."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-shared",
                               "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        vp = ctypes.c_void_p
        L.oracle_mix.argtypes, L.oracle_mix.restype = [u64], u64
        L.oracle_hash_bytes.argtypes, L.oracle_hash_bytes.restype = [vp, u64, u64], u64
        L.oracle_page_hash.argtypes, L.oracle_page_hash.restype = [vp, u64], u64
        L.oracle_pages_of.argtypes, L.oracle_pages_of.restype = [u64], u64
        L.oracle_valid_bytes.argtypes, L.oracle_valid_bytes.restype = [u64, u64], u64
        L.oracle_total_pages.argtypes, L.oracle_total_pages.restype = [vp, u32], u64
        L.oracle_hash_all.argtypes, L.oracle_hash_all.restype = [vp, vp, u32, vp], None
        L.oracle_dirty.argtypes, L.oracle_dirty.restype = [vp, vp, vp, i32, u64, vp], u64
        L.oracle_verify.argtypes, L.oracle_verify.restype = [vp, vp, vp, u32, vp], u64
        L.oracle_image_size.argtypes, L.oracle_image_size.restype = [u32, u64], u64
        L.oracle_build_image.argtypes = [vp, vp, vp, u32, vp, vp, i32, u64, u64, vp, u64]
        L.oracle_build_image.restype = u64
        L.oracle_check_image.argtypes, L.oracle_check_image.restype = [vp, u64], i32
        L.oracle_apply_image.argtypes = [vp, u64, vp, vp, u32, vp]
        L.oracle_apply_image.restype = i32
        L.oracle_bpd_encode.argtypes, L.oracle_bpd_encode.restype = [vp, vp], u64
        L.oracle_bpd_decode.argtypes, L.oracle_bpd_decode.restype = [vp, u64, vp], i32
        L.oracle_build_cimage.argtypes = [vp, vp, vp, u32, vp, vp, i32, u64, u64, vp, vp, vp, u64]
        L.oracle_build_cimage.restype = u64
        L.oracle_check_cimage.argtypes, L.oracle_check_cimage.restype = [vp, u64], i32
        L.oracle_apply_cimage.argtypes = [vp, u64, vp, vp, u32, vp, vp]
        L.oracle_apply_cimage.restype = i32
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    # callers keep `a` alive in a local across the C call
    return a.ctypes.data


def _ptr_array(arrays: Sequence[np.ndarray]) -> np.ndarray:
    return np.array([a.ctypes.data for a in arrays], dtype=np.uint64)


def _u8(a) -> np.ndarray:
    a = np.asarray(a)
    assert a.flags["C_CONTIGUOUS"]
    return a.view(np.uint8).reshape(-1)


def mix(z: int) -> int:
    return int(lib().oracle_mix(z))


def hash_bytes(buf, first_index: int = 0) -> int:
    b = _u8(np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray)) else buf)
    return int(lib().oracle_hash_bytes(_ptr(b), b.size, first_index))


def page_hash(buf) -> int:
    b = _u8(np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray)) else buf)
    assert b.size <= PAGE
    return int(lib().oracle_page_hash(_ptr(b), b.size))


def pages_of(nbytes: int) -> int:
    return int(lib().oracle_pages_of(nbytes))


def valid_bytes(nbytes: int, page: int) -> int:
    return int(lib().oracle_valid_bytes(nbytes, page))


def total_pages(sizes: Sequence[int]) -> int:
    s = np.asarray(sizes, dtype=np.uint64)
    return int(lib().oracle_total_pages(_ptr(s), s.size))


def hash_all(allocs: Sequence[np.ndarray]) -> np.ndarray:
    """Page hashes of every page of every allocation, in global page order."""
    allocs = [_u8(a) for a in allocs]
    ptrs = _ptr_array(allocs)
    sizes = np.array([a.size for a in allocs], dtype=np.uint64)
    out = np.zeros(total_pages(sizes), dtype=np.uint64)
    lib().oracle_hash_all(_ptr(ptrs), _ptr(sizes), len(allocs), _ptr(out))
    return out


def dirty(h: np.ndarray, h_prev: np.ndarray, force: np.ndarray | None, full: bool):
    h = np.ascontiguousarray(h, dtype=np.uint64)
    h_prev = np.ascontiguousarray(h_prev, dtype=np.uint64)
    out = np.zeros(h.size, dtype=np.uint8)
    fp = None
    if force is not None:
        force = np.ascontiguousarray(force, dtype=np.uint8)
        fp = _ptr(force)
    n = lib().oracle_dirty(_ptr(h), _ptr(h_prev), fp, int(bool(full)), h.size, _ptr(out))
    return out, int(n)


def verify(allocs, prev_allocs, dirty_flags: np.ndarray):
    """Exact compare of hash-clean pages; returns (dirty, collisions)."""
    allocs = [_u8(a) for a in allocs]
    prev_allocs = [_u8(a) for a in prev_allocs]
    sizes = np.array([a.size for a in allocs], dtype=np.uint64)
    d = np.array(dirty_flags, dtype=np.uint8, copy=True)
    ptrs, prev_ptrs = _ptr_array(allocs), _ptr_array(prev_allocs)
    n = lib().oracle_verify(_ptr(ptrs), _ptr(prev_ptrs), _ptr(sizes), len(allocs), _ptr(d))
    return d, int(n)


def image_size(n_allocs: int, n_dirty: int) -> int:
    return int(lib().oracle_image_size(n_allocs, n_dirty))


def bpd_encode(slot) -> bytes:
    """Byte-plane dictionary code of one 65,536-byte slot (65,536 bytes back
    means stored as is)."""
    b = _u8(np.frombuffer(slot, dtype=np.uint8) if isinstance(slot, (bytes, bytearray)) else slot)
    assert b.size == PAGE
    out = np.zeros(PAGE, dtype=np.uint8)
    n = int(lib().oracle_bpd_encode(_ptr(b), _ptr(out)))
    return out[:n].tobytes()


def bpd_decode(enc: bytes):
    """(status, 65,536-byte slot) of an encoded slot."""
    b = np.frombuffer(enc, dtype=np.uint8)
    out = np.zeros(PAGE, dtype=np.uint8)
    st = int(lib().oracle_bpd_decode(_ptr(b) if b.size else 0, b.size, _ptr(out)))
    return st, out.tobytes()


def image_version(img) -> int:
    return int(np.frombuffer(img[8:12], dtype=np.uint32)[0])


def build_image(allocs, ids, h, dirty_flags, full: bool, seq: int, parent_seq: int,
                compress: bool = False) -> bytes:
    if compress:
        return build_cimage(allocs, ids, h, dirty_flags, full, seq, parent_seq)
    allocs = [_u8(a) for a in allocs]
    sizes = np.array([a.size for a in allocs], dtype=np.uint64)
    ids = np.asarray(ids, dtype=np.uint32)
    h = np.ascontiguousarray(h, dtype=np.uint64)
    d = np.ascontiguousarray(dirty_flags, dtype=np.uint8)
    size = image_size(len(allocs), int(d.astype(np.uint64).sum()))
    out = np.zeros(size, dtype=np.uint8)
    ptrs = _ptr_array(allocs)
    got = lib().oracle_build_image(_ptr(ptrs), _ptr(sizes), _ptr(ids), len(allocs),
                                   _ptr(h), _ptr(d), int(bool(full)), seq, parent_seq,
                                   _ptr(out), size)
    assert got == size
    return out.tobytes()


def build_cimage(allocs, ids, h, dirty_flags, full: bool, seq: int, parent_seq: int) -> bytes:
    """The compressed (version 2) image of the dirty pages."""
    allocs = [_u8(a) for a in allocs]
    sizes = np.array([a.size for a in allocs], dtype=np.uint64)
    ids = np.asarray(ids, dtype=np.uint32)
    h = np.ascontiguousarray(h, dtype=np.uint64)
    d = np.ascontiguousarray(dirty_flags, dtype=np.uint8)
    n = int(d.astype(np.uint64).sum())
    scratch = np.zeros(max(n, 1) * PAGE, dtype=np.uint8)
    lens = np.zeros(max(n, 1), dtype=np.uint64)
    ptrs = _ptr_array(allocs)
    args = (_ptr(ptrs), _ptr(sizes), _ptr(ids), len(allocs), _ptr(h), _ptr(d), int(bool(full)),
            seq, parent_seq, _ptr(scratch), _ptr(lens))
    size = int(lib().oracle_build_cimage(*args, None, 0))
    out = np.zeros(size, dtype=np.uint8)
    got = lib().oracle_build_cimage(*args, _ptr(out), size)
    assert got == size
    return out.tobytes()


def check_image(img) -> int:
    b = np.frombuffer(img, dtype=np.uint8)
    if b.size >= 12 and image_version(img) == 2:
        return int(lib().oracle_check_cimage(_ptr(b), b.size))
    return int(lib().oracle_check_image(_ptr(b), b.size))


def apply_image(img, allocs, h_prev: np.ndarray | None) -> int:
    """Restore one image onto writable host arrays; updates h_prev in place."""
    b = np.frombuffer(img, dtype=np.uint8)
    if b.size >= 12 and image_version(img) == 2:
        allocs = [_u8(a) for a in allocs]
        sizes = np.array([a.size for a in allocs], dtype=np.uint64)
        hp = None
        if h_prev is not None:
            assert h_prev.dtype == np.uint64 and h_prev.flags["C_CONTIGUOUS"]
            hp = _ptr(h_prev)
        n = int(np.frombuffer(img[40:48], dtype=np.uint64)[0])
        scratch = np.zeros(max(n, 1) * PAGE, dtype=np.uint8)
        ptrs = _ptr_array(allocs)
        return int(lib().oracle_apply_cimage(_ptr(b), b.size, _ptr(ptrs), _ptr(sizes),
                                             len(allocs), hp, _ptr(scratch)))
    allocs = [_u8(a) for a in allocs]
    sizes = np.array([a.size for a in allocs], dtype=np.uint64)
    hp = None
    if h_prev is not None:
        assert h_prev.dtype == np.uint64 and h_prev.flags["C_CONTIGUOUS"]
        hp = _ptr(h_prev)
    ptrs = _ptr_array(allocs)
    return int(lib().oracle_apply_image(_ptr(b), b.size, _ptr(ptrs), _ptr(sizes),
                                        len(allocs), hp))


class OracleSet:
    """A registered set as the oracle sees it: host copies, hash table, seq.

    Mirrors the life cycle of a checkpointed set: ``checkpoint`` hashes all
    pages, applies the dirty rule (first checkpoint after registration is
    all dirty), writes the image and commits the hashes; ``restore`` applies
    a chain base-to-end and installs the image hashes.
    """

    def __init__(self, sizes: Sequence[int], ids: Sequence[int] | None = None,
                 compress: bool = False):
        self.compress = compress
        self.sizes = [int(s) for s in sizes]
        self.ids = list(ids) if ids is not None else list(range(len(self.sizes)))
        self.next_id = max(self.ids) + 1 if self.ids else 0
        n = total_pages(self.sizes)
        self.h_prev = np.zeros(n, dtype=np.uint64)
        self.force = np.ones(n, dtype=np.uint8)
        self.seq = 0
        self.last_seq = None
        self.new_base = True

    def _registration_changed(self):
        # Algorithm 1: a region that starts being tracked has every page
        # dirty.  Page indices of an image refer to the allocation table of
        # its chain, so any change of the table starts a new chain: the next
        # image is full (no parent), while sequence numbers keep counting.
        n = total_pages(self.sizes)
        self.h_prev = np.zeros(n, dtype=np.uint64)
        self.force = np.ones(n, dtype=np.uint8)
        self.new_base = True

    def register(self, size: int) -> int:
        """Add an allocation at the end of the registration order; returns
        its id (ids count up from the set's first and are never reused)."""
        self.sizes.append(int(size))
        self.ids.append(self.next_id)
        self.next_id += 1
        self._registration_changed()
        return self.ids[-1]

    def unregister(self, alloc_id: int) -> None:
        """Drop an allocation; the others keep their order and ids."""
        k = self.ids.index(alloc_id)
        del self.sizes[k]
        del self.ids[k]
        self._registration_changed()

    def checkpoint(self, allocs, full: bool = False, verify_prev=None):
        h = hash_all(allocs)
        d, n = dirty(h, self.h_prev, self.force, full)
        collisions = 0
        if verify_prev is not None:
            d, collisions = verify(allocs, verify_prev, d)
        parent = self.last_seq if self.last_seq is not None else 0xFFFFFFFFFFFFFFFF
        is_full = full or self.new_base
        img = build_image(allocs, self.ids, h, d, is_full, self.seq, parent, self.compress)
        self.h_prev = h
        self.force[:] = 0
        self.new_base = False
        self.last_seq = self.seq
        self.seq += 1
        return img, d, h, collisions

    def restore(self, chain, allocs) -> int:
        for img in chain:
            st = apply_image(img, allocs, self.h_prev)
            if st != OK:
                return st
        self.force[:] = 0
        self.new_base = False
        last = chain[-1]
        self.last_seq = int(np.frombuffer(last[16:24], dtype=np.uint64)[0])
        self.seq = self.last_seq + 1
        return OK
