"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no page hash, no dirty rule, no image format).  Both
the CUDA path and the CPU oracle consume what it produces: device tensors
filled here are copied to the host for the oracle.

Workload recipes (the paper's own applications and data are not used;
synthetic data of the same shape stands in for them):

* ``small16m``  one 16 MiB fp32 allocation, uniform in [-1, 1) (the synthetic
  single-GPU benchmark's random-float vectors, Section 4.4, scaled down);
  10 % of pages rewritten, chosen uniformly without replacement.
* ``uint32_8g`` one 8 GiB allocation of random 32-bit words; 5 % of pages
  (6,554) dirtied per step in clustered runs: run starts uniform, run
  lengths geometric with p = 1/16 truncated to [1, 64], runs merged until
  the union reaches the target, the last run trimmed to hit it exactly.
* ``stencil``   200 fp64 fields with log-uniform sizes (4 KiB .. 512 MiB,
  rounded to 4 KiB, rescaled to a target total), the many-regions-of-uneven-
  size shape of the HPGMG/HYPRE runs (Section 4.2).
* ``large``     4,096 allocations, log-uniform 64 KiB .. 2 GiB rescaled to a
  target total, fp32 or bf16 bit patterns, 2 % of pages per step.

A "mutation" xors every 64-bit word of a chosen page with one nonzero
per-page mask, so every chosen page really changes.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

PAGE = 65536
KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30


def pages_of(nbytes: int) -> int:
    return -(-nbytes // PAGE)


@dataclass
class Workload:
    name: str
    sizes: List[int]
    kind: str
    dirty_frac: float
    steps: int
    dirty_mode: str = "uniform"  # uniform | runs
    seed: int = 0x5EED
    meta: dict = field(default_factory=dict)

    @property
    def total_bytes(self) -> int:
        return sum(self.sizes)

    @property
    def n_pages(self) -> int:
        return sum(pages_of(s) for s in self.sizes)


def loguniform_sizes(seed: int, n: int, lo: int, hi: int, total, round_to: int = 4 * KiB,
                     tol: float = 0.005) -> List[int]:
    """n sizes log-uniform in [lo, hi], rounded to `round_to`; with a `total`,
    then rescaled by a common factor (clamped to [lo, hi]) until the sum is
    within `tol` of it."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))
    if total is None:
        return [int(v) for v in np.clip(np.round(x / round_to) * round_to, lo, hi)]
    for _ in range(200):
        s = np.clip(np.round(x / round_to) * round_to, lo, hi)
        t = float(s.sum())
        if abs(t - total) <= tol * total:
            break
        x = np.clip(x * (total / t), lo, hi)
    return [int(v) for v in s]


def workload(name: str) -> Workload:
    if name == "small16m":
        return Workload(name, [16 * MiB], "fp32", 0.10, 1, "uniform", 0x5EED + 0)
    if name == "uint32_8g":
        return Workload(name, [8 * GiB], "u32", 0.05, 10, "runs", 0x5EED + 1)
    if name == "stencil":
        sizes = loguniform_sizes(0x5EED + 2, 200, 4 * KiB, 512 * MiB, 24 * GiB)
        return Workload(name, sizes, "fp64", 0.30, 20, "stencil", 0x5EED + 2)
    if name == "large":
        sizes = loguniform_sizes(0x5EED + 4, 4096, 64 * KiB, 2 * GiB, 140 * GiB)
        return Workload(name, sizes, "fp32", 0.02, 50, "uniform", 0x5EED + 4)
    if name == "oversub":
        # Section 4.4's synthetic benchmark: two vectors of 2^32 fp32 (32 GiB)
        # in managed memory, twice what its GPU holds
        return Workload(name, [4 * GiB * 4, 4 * GiB * 4], "fp32", 0.02, 10, "uniform", 0x5EED + 5,
                        {"device_holds_bytes": 16 * GiB})
    if name == "serving":
        # 32 clients, footprints log-uniform 1 MiB .. 4 GiB (not rescaled);
        # the mean of the per-request U[1 %, 50 %] rewrite as the dirty share
        sizes = loguniform_sizes(0x5EED + 3, 32, 1 * MiB, 4 * GiB, None, round_to=PAGE)
        return Workload(name, sizes, "u32", 0.255, 2000, "uniform", 0x5EED + 3)
    raise KeyError(name)


# ------------------------------------------------------------- selections ---

def choose_uniform(seed: int, n_pages: int, k: int) -> np.ndarray:
    """k distinct page indices in [0, n_pages), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_pages, size=min(k, n_pages), replace=False)).astype(np.int64)


def choose_runs(seed: int, n_pages: int, target: int, p: float = 1 / 16, max_len: int = 64) -> np.ndarray:
    """Clustered dirty runs: uniform starts, geometric(p) lengths truncated to
    [1, max_len], merged until `target` distinct pages; sorted."""
    rng = np.random.default_rng(seed)
    target = min(target, n_pages)
    chosen = np.zeros(n_pages, dtype=bool)
    count = 0
    while count < target:
        start = int(rng.integers(0, n_pages))
        length = int(min(max(rng.geometric(p), 1), max_len))
        seg = chosen[start:start + length]
        new = np.flatnonzero(~seg)
        if count + new.size > target:
            new = new[: target - count]
        seg[new] = True
        count += new.size
    return np.flatnonzero(chosen).astype(np.int64)


def choose_step(wl: Workload, step: int, n_pages: int) -> np.ndarray:
    k = max(1, int(round(wl.dirty_frac * n_pages)))
    seed = wl.seed * 1_000_003 + step
    if wl.dirty_mode == "runs":
        return choose_runs(seed, n_pages, k)
    return choose_uniform(seed, n_pages, k)


# ------------------------------------------------------------ device fills ---

def _torch():
    import torch
    return torch


def fill_(buf, seed: int, kind: str) -> None:
    """Fill a uint8 tensor in place from a seeded torch generator."""
    torch = _torch()
    g = torch.Generator(device=buf.device)
    g.manual_seed(seed)
    n = buf.numel()
    n8 = n // 8 * 8
    if kind in ("fp32", "fp64") and n8:
        dt = torch.float32 if kind == "fp32" else torch.float64
        buf[:n8].view(dt).uniform_(-1.0, 1.0, generator=g)
    elif kind == "bf16" and n8:
        buf[:n8].view(torch.bfloat16).normal_(generator=g)
    elif n8:
        buf[:n8].view(torch.int64).random_(generator=g)
    if n > n8:
        buf[n8:] = torch.randint(0, 256, (n - n8,), dtype=torch.uint8, device=buf.device, generator=g)


STENCIL_NX = STENCIL_NY = 64  # fp64 box planes of 64 x 64 (32 KiB, two per page)


def stencil_plan(nbytes: int, frac: float, seed: int):
    """Interior z-range [z0, z0 + L) of an fp64 (nz, 64, 64) box so that about
    `frac` of the box's planes are rewritten; None if the box is too thin."""
    nz = nbytes // (8 * STENCIL_NX * STENCIL_NY)
    if nz < 3:
        return None
    L = max(1, min(nz - 2, int(round(frac * nz))))
    rng = np.random.default_rng(seed)
    z0 = int(rng.integers(1, nz - L)) if nz - L > 1 else 1
    return nz, z0, L


def stencil_step_(buf, plan) -> None:
    """27-point average (3x3x3 box mean) over the interior sub-box
    z in [z0, z0+L), y, x in [1, 63) of an fp64 (nz, 64, 64) field, written
    in place: the synthetic stencil application's update."""
    if plan is None:
        return
    torch = _torch()
    nz, z0, L = plan
    box = buf[: nz * 8 * STENCIL_NX * STENCIL_NY].view(torch.float64).view(nz, STENCIL_NY, STENCIL_NX)
    src = box[z0 - 1: z0 + L + 1].unsqueeze(0).unsqueeze(0)
    avg = torch.nn.functional.avg_pool3d(src, kernel_size=3, stride=1)
    box[z0: z0 + L, 1: STENCIL_NY - 1, 1: STENCIL_NX - 1] = avg[0, 0]


def mutate_pages_(buf, pages, seed: int, has_tail=None) -> None:
    """xor every word of each listed page (page indices within `buf`) with a
    per-page nonzero 64-bit mask; a partial last page gets a nonzero byte mask.

    `pages` is a host sequence, or a device tensor of whole-page indices with
    `has_tail` saying whether the partial last page is also chosen (this form
    never waits for the device)."""
    torch = _torch()
    n = buf.numel()
    n_full = n // PAGE
    if isinstance(pages, torch.Tensor):
        full = pages.to(device=buf.device, dtype=torch.int64)
        tail = bool(has_tail) and n > n_full * PAGE
    else:
        p = np.asarray(pages, dtype=np.int64)
        tail = bool((p == n_full).any()) and n > n_full * PAGE
        full = torch.as_tensor(p[p < n_full], device=buf.device)
    g = torch.Generator(device=buf.device)
    g.manual_seed(seed)
    if full.numel():
        v = buf[: n_full * PAGE].view(torch.int64).view(n_full, PAGE // 8)
        masks = torch.randint(1, 2**62, (full.numel(), 1), dtype=torch.int64, device=buf.device,
                              generator=g) | 1
        v[full] = v[full] ^ masks
    if tail:
        m = torch.randint(1, 256, (1,), dtype=torch.int64, device=buf.device, generator=g).to(torch.uint8)
        buf[n_full * PAGE:].bitwise_xor_(m)


# ----------------------------------------------------- managed memory -------
#
# The paper's applications keep their data in CUDA managed (unified) memory.
# `managed_empty` makes such an allocation with the CUDA runtime, asks for
# its pages to sit on the device (as they do after a kernel has touched
# them), and returns a uint8 tensor over it; the allocation is freed when the
# last tensor viewing it goes away.

class _CudaMemLocation(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("id", ctypes.c_int)]


_cudart = None


def _rt():
    global _cudart
    if _cudart is None:
        rt = ctypes.CDLL("libcudart.so.13")
        rt.cudaMallocManaged.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_uint]
        rt.cudaMemPrefetchAsync.argtypes = [ctypes.c_void_p, ctypes.c_size_t, _CudaMemLocation,
                                            ctypes.c_uint, ctypes.c_void_p]
        rt.cudaFree.argtypes = [ctypes.c_void_p]
        rt.cudaStreamSynchronize.argtypes = [ctypes.c_void_p]
        _cudart = rt
    return _cudart


class _Managed:
    """Owner of one managed allocation, exported to torch by the CUDA array
    interface (torch keeps this object alive as long as the tensor)."""

    def __init__(self, nbytes: int, device: int, where: str):
        rt = _rt()
        p = ctypes.c_void_p()
        if rt.cudaMallocManaged(ctypes.byref(p), nbytes, 1) != 0:  # cudaMemAttachGlobal
            raise MemoryError(f"cudaMallocManaged({nbytes}) failed")
        self.ptr, self.nbytes = p.value, nbytes
        try:
            managed_prefetch(self.ptr, nbytes, where, device)
        except RuntimeError:
            rt.cudaFree(self.ptr)
            self.ptr = None
            raise
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1",
                                         "data": (self.ptr, False), "version": 3, "strides": None}

    def __del__(self):
        if getattr(self, "ptr", None):
            _rt().cudaFree(self.ptr)
            self.ptr = None


def managed_prefetch(ptr: int, nbytes: int, where: str, device: int = 0) -> None:
    """Move managed pages to the device or the host (synchronous)."""
    rt = _rt()
    # cudaMemLocationTypeDevice = 1, cudaMemLocationTypeHost = 2
    loc = _CudaMemLocation(1, device) if where == "device" else _CudaMemLocation(2, 0)
    if rt.cudaMemPrefetchAsync(ptr, nbytes, loc, 0, None) != 0 or rt.cudaStreamSynchronize(None) != 0:
        raise RuntimeError("cudaMemPrefetchAsync failed")


def managed_advise(ptr: int, nbytes: int, advice: str, device: int = 0) -> None:
    """cudaMemAdvise on a managed range: "preferred_host" (preferred location
    the host) or "accessed_by" (the device keeps a mapping), as an
    application sets it."""
    rt = _rt()
    rt.cudaMemAdvise.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, _CudaMemLocation]
    code, loc = {"preferred_host": (3, _CudaMemLocation(2, 0)),
                 "accessed_by": (5, _CudaMemLocation(1, device))}[advice]
    if rt.cudaMemAdvise(ptr, nbytes, code, loc) != 0:
        raise RuntimeError("cudaMemAdvise failed")


def managed_accessed_by(ptr: int, nbytes: int) -> list:
    """Devices holding cudaMemAdviseSetAccessedBy for the whole range."""
    rt = _rt()
    rt.cudaMemRangeGetAttribute.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_size_t]
    devs = (ctypes.c_int * 64)(*([-2] * 64))
    if rt.cudaMemRangeGetAttribute(devs, ctypes.sizeof(devs), 3, ptr, nbytes) != 0:
        raise RuntimeError("cudaMemRangeGetAttribute failed")
    return [d for d in devs if d >= 0]


def managed_empty(nbytes: int, device: int = 0, where: str = "device"):
    """uint8 CUDA tensor over a new managed allocation whose pages were
    prefetched to `where` ("device" or "host")."""
    t = _torch()
    return t.as_tensor(_Managed(nbytes, device, where), device=f"cuda:{device}")
