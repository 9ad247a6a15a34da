#!/usr/bin/env python
"""Benchmark of the B300 capture/restore path (one JSON line on rank 0).

Workload (default ``large``): 140 GiB of managed memory (cudaMallocManaged,
pages prefetched to the device) holding fp32 data, carved into 4,096
allocations with sizes log-uniform 64 KiB .. 2 GiB, 64 KiB pages
(2,295,728).  Setup takes the full checkpoint (its payload crosses the link
and is dropped: a 140 GiB image does not fit the host beside its
incrementals) and autotunes the thread mappings; each step then lets the
application's scatter kernel rewrite 2 % of the pages (45,915, chosen
uniformly) and takes an incremental checkpoint on the application's
stream, launched as one CUDA graph.  A step is one pass of the whole path:
hash every page, detect dirty pages, compact them into staging and drain
them over the host link (null sink); the drain overlaps the next step's
application work and capture.

``value`` is the capture throughput: footprint bytes checkpointed per
second of capture-kernel device time (hash + scan + gather, CUDA events on
the capture stream), mean over the K timed steps.  ``ms_per_step`` is the
whole step (application update, capture, drain) bracketed by a barrier and
a synchronize.  Inputs (140 GiB) are larger than L2 (126 MB), so no flush is
needed between steps.  ``e2e`` is the public API end to end with host
buffers (the step's new page contents uploaded from pinned memory, the
image read back into host memory).  ``--workload uint32_8g`` measures the
8 GiB single-allocation workload (memory sink, chain restore, verify mode).

``--impl reference`` times the CPU oracle (test infrastructure, single
thread, and beside it the same oracle calls on every host core) on a
bounded sample of the same workload: the paper has no code to run, so the
oracle is the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("checkpoint capture GB/s vs HBM peak; drain GB/s vs host link; "
          "p50/p99 ckpt latency")
UNIT = "GB/s"
FALLBACK_HBM_GBS = 6400.0
NOMINAL_LINK_GBS = 63.0  # PCIe Gen5 x16 per direction


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large",
                    help="large (default: 140 GiB of managed fp32 in 4,096 allocations), "
                         "uint32_8g, small16m, stencil, serving or oversub")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-verify", action="store_true", help="skip the verify-mode measurement")
    ap.add_argument("--no-restore", action="store_true",
                    help="large workload: skip the chain restore of a 40 GiB prefix")
    ap.add_argument("--compress", action="store_true",
                    help="images in the compressed form (byte-plane dictionary code on the device)")
    ap.add_argument("--managed-in-place", action="store_true",
                    help="stencil/large: sets look up managed placement at every checkpoint "
                         "(managed_in_place=1)")
    ap.add_argument("--kind", choices=["u32", "fp32", "fp64", "bf16"], default=None,
                    help="element kind of the synthetic data (uint32, stencil and large workloads)")
    ap.add_argument("--sink", choices=["memory", "file"], default="memory",
                    help="uint32 workload: where the writer persists images (file: a "
                         "temporary directory on the host's disk, fsync per image)")
    ap.add_argument("--cpu-sample-mib", type=int, default=2048,
                    help="size of the workload sample the CPU oracle is timed on")
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: request count")
    ap.add_argument("--mapping", default="",
                    help="'H,G': fixed hash and gather thread mappings instead of the autotuner")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: launch each capture as one CUDA graph (0: one launch per op)")
    ap.add_argument("--footprint-gib", type=int, default=0,
                    help="resize the uint32 workload (one allocation) or the large workload "
                         "(4,096 allocations rescaled to this total): small profiling cases")
    ap.add_argument("--memory", choices=["device", "managed"], default=None,
                    help="application memory: cudaMalloc (PyTorch) or cudaMallocManaged "
                         "prefetched to the device; default managed for the large workload")
    return ap.parse_args(argv)


def bench_workload(args):
    """The workload a run measures, with --footprint-gib and --kind applied."""
    from paper_1808_00117_b300 import workloads as W
    wl = W.workload(args.workload)
    if args.footprint_gib and wl.name == "large":
        wl.sizes = W.loguniform_sizes(wl.seed, len(wl.sizes), 64 * W.KiB, 2 * W.GiB,
                                      args.footprint_gib * W.GiB)
        wl.meta["resized_gib"] = args.footprint_gib
    elif args.footprint_gib:
        wl.sizes = [args.footprint_gib * W.GiB]
        wl.name = f"uint32_{args.footprint_gib}g"
    if args.kind:
        wl.kind = args.kind
    return wl


def host_budget_bytes() -> int:
    """Host memory one rank may pin for images: 60 % of the node's available
    memory, shared by the ranks on the node."""
    avail = 0
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    if not avail:
        avail = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    ranks = int(os.environ.get("LOCAL_WORLD_SIZE", os.environ.get("WORLD_SIZE", "1")))
    return int(0.6 * avail / max(1, ranks))


def raw_image_bytes(info) -> int:
    """Bytes of the uncompressed image with the same pages."""
    return 64 + 16 * info["n_allocs"] + 16 * info["n_dirty"] + info["n_dirty"] * 65536 + 8


def app_memory(args, wl) -> str:
    return args.memory or ("managed" if wl.name == "large" else "device")


def app_alloc(torch, kind: str, nbytes: int, dev):
    """The application's allocation: device memory or managed memory whose
    pages sit on the device."""
    from paper_1808_00117_b300 import workloads as W
    if kind == "managed":
        return W.managed_empty(nbytes, device=dev.index if dev.index is not None else 0)
    return torch.empty(nbytes, dtype=torch.uint8, device=dev)


MEMORY_DESC = {"device": "device memory (cudaMalloc through PyTorch)",
               "managed": "managed memory (cudaMallocManaged, pages prefetched to the device)"}


# ------------------------------------------------------------ distributed ---

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float, device=None) -> float:
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float, device=None) -> float:
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while work runs."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 20):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="crum_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", f"-lms={self.period}"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def mark(self, which: str):
        setattr(self, which, time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import datetime
        rows, all_rows = [], []
        t0, t1 = getattr(self, "t0", None), getattr(self, "t1", None)
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    row = (float(parts[2]), float(parts[3]), parts[5:10])
                except ValueError:
                    continue
                all_rows.append(row)
                if t0 is None or (t0 - 0.05 <= ts <= (t1 or ts) + 0.05):
                    rows.append(row)
        os.unlink(self.path)
        if not rows:
            rows = all_rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, r in rows:
            for n, v in zip(names, r[1:]):
                if v.lower() == "active":
                    reasons.add(n)
        busy = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return {"hbm_gbs": float(mp["hbm_gbs"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS, "source": "fallback"}


def kernel_code_digest() -> str:
    """First 16 hex digits of the sha256 of the capture kernels' code
    (kernels.cu with its headers kernels.h, launch.cuh and device.cuh) with
    comments and whitespace removed, so that editing a comment, or the
    compression and restore kernels, keeps a recorded profile of a capture
    kernel valid, and editing its code does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in ("kernels.cu", "kernels.h", "launch.cuh", "device.cuh"):
        text = open(os.path.join(ROOT, "paper_1808_00117_b300", "csrc", name)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel: str, workload: str):
    """DRAM bytes per launch recorded from ncu in profiles/, if the recorded
    device-code digest still matches the code being benchmarked."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
        digest = kernel_code_digest()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("device_code_sha256_16") != digest:
        return None
    try:
        return int(vals["traffic_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------- CPU arm ---

def oracle_sample(wl, sample_mib: int):
    """The bounded sample of a workload that the oracle is timed on: the
    workload's allocations taken in registration order while they fit in
    `sample_mib` MiB (the first `sample_mib` MiB of a one-allocation
    workload), filled on the host from a numpy generator with the workload's
    element kind.  Returns (sizes, host arrays)."""
    budget = sample_mib << 20
    if len(wl.sizes) == 1:
        sizes = [min(wl.sizes[0], budget)]
    else:
        sizes, tot = [], 0
        for n in wl.sizes:
            if tot + n <= budget:
                sizes.append(int(n))
                tot += n
        if not sizes:
            sizes = [int(min(wl.sizes))]
    rng = np.random.default_rng(wl.seed)
    allocs = []
    for n in sizes:
        if wl.kind == "fp32":
            a = (rng.random(n // 4, dtype=np.float32) * 2 - 1).view(np.uint8)
        elif wl.kind == "fp64":
            a = (rng.random(n // 8) * 2 - 1).view(np.uint8)
        else:
            a = rng.integers(0, 2**32, size=n // 4, dtype=np.uint32).view(np.uint8)
        allocs.append(np.ascontiguousarray(a))
    return sizes, allocs


def oracle_cpu_baseline(wl, sample_mib: int, steps: int, warmup: int, compress: bool = False):
    """Time the CPU oracle's incremental checkpoint on a bounded sample of
    the workload (`oracle_sample`), the workload's dirty share of pages
    rewritten per step (each word of a chosen page xored with a nonzero
    mask), in two forms:

    - single thread: ``OracleSet.checkpoint`` as it stands (hash every page,
      dirty rule, image with its trailer);
    - all cores: the same oracle calls, with the page hashes (every byte of
      the footprint is read; the image holds the dirty share) taken on
      page-aligned slices by one host thread per core (the C calls release
      the interpreter lock), then the oracle's dirty rule and image writer
      on one thread.  Its image must equal the single-thread image byte for
      byte at every step.

    With `compress` the images are the compressed form (the oracle's codec
    on every dirty page), as the GPU arm's are with --compress.
    """
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    from paper_1808_00117_b300 import workloads as W
    sizes, allocs = oracle_sample(wl, sample_mib)
    S = sum(sizes)
    pages = [W.pages_of(n) for n in sizes]
    first = np.cumsum([0] + pages)
    n_pages = int(first[-1])
    words = [a.view(np.uint64) for a in allocs]
    o = oracle.OracleSet(sizes, compress=compress)
    o.checkpoint(allocs)  # the full base, untimed
    cores = len(os.sched_getaffinity(0))
    span = 256  # pages per slice (16 MiB): many slices per thread for balance
    slices = [allocs[i][p * W.PAGE:min((p + span) * W.PAGE, sizes[i])]
              for i in range(len(sizes)) for p in range(0, pages[i], span)]
    h_prev, seq, last = o.h_prev.copy(), o.seq, o.last_seq
    rng = np.random.default_rng(wl.seed + 1)
    t1, tn = [], []
    with ThreadPoolExecutor(max_workers=cores) as ex:
        for step in range(warmup + steps):
            chosen = W.choose_step(wl, 1000 + step, n_pages)
            masks = rng.integers(1, 2**62, size=chosen.size, dtype=np.uint64) | np.uint64(1)
            for g, m in zip(chosen.tolist(), masks):
                i = int(np.searchsorted(first, g, side="right")) - 1
                p = g - int(first[i])
                words[i][p * (W.PAGE // 8):(p + 1) * (W.PAGE // 8)] ^= m
            a0 = time.perf_counter()
            img, d, _, _ = o.checkpoint(allocs)
            a1 = time.perf_counter()
            h = np.concatenate(list(ex.map(lambda x: oracle.hash_all([x]), slices)))
            dn, _ = oracle.dirty(h, h_prev, None, False)
            img_n = oracle.build_image(allocs, list(range(len(sizes))), h, dn, False, seq, last,
                                       compress)
            a2 = time.perf_counter()
            assert int(d.sum()) == chosen.size, "oracle dirty count differs from the rewrite"
            assert img_n == img, "all-core oracle image differs from the single-thread image"
            h_prev, last, seq = h, seq, seq + 1
            if step >= warmup:
                t1.append(a1 - a0)
                tn.append(a2 - a1)
    k = int(round(wl.dirty_frac * n_pages))
    sample = (f"{len(sizes)} allocation(s), {S / 2**20:.0f} MiB of the {wl.name} workload "
              f"({n_pages} pages, {k} rewritten per step), {steps} incremental checkpoints"
              + (", compressed images" if compress else ""))
    m1, mn = statistics.mean(t1), statistics.mean(tn)
    return {"value": S / m1 / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": sample + ", single-thread C oracle",
            "ms_per_checkpoint": m1 * 1e3, "sample_bytes": S,
            "all_cores": {"value": round(S / mn / 1e9, 3), "unit": UNIT, "cores": cores,
                          "kind": "oracle", "ms_per_checkpoint": round(mn * 1e3, 3),
                          "image_equal_to_single_thread": True,
                          "sample": sample + f": page hashes on {len(slices)} page-aligned "
                                    f"slices, one thread per core; dirty rule and image "
                                    f"writer on one thread"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = bench_workload(args)
    t0 = time.perf_counter()
    cb = oracle_cpu_baseline(wl, args.cpu_sample_mib, args.steps, args.warmup, bool(args.compress))
    wall = time.perf_counter() - t0
    line = {
        "impl": "reference", "metric": METRIC, "value": round(cb["value"], 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(cb["ms_per_checkpoint"], 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.name, "sample_bytes": cb["sample_bytes"],
                   "parallelism": "single host thread"},
        "cpu_baseline": {**{k: cb[k] for k in ("unit", "cores", "kind", "sample")},
                         "value": round(cb["value"], 4), "all_cores": cb["all_cores"]},
        "e2e": {"value": round(cb["value"], 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": round(wall, 2),
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm ---

def pct(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if xs else None


def link_d2h_peak(torch, nbytes=2 << 30):
    """Pinned device->host copy bandwidth, measured with CUDA events."""
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    for _ in range(2):
        host.copy_(dev, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        host.copy_(dev, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    gbs = 3 * nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del dev, host
    return gbs


def link_h2d_peak(torch, nbytes=2 << 30):
    """Pinned host->device copy bandwidth, measured with CUDA events."""
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    for _ in range(2):
        dev.copy_(host, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        dev.copy_(host, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    gbs = 3 * nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del dev, host
    return gbs


def link_bidir_peak(torch, nbytes=1 << 30, reps=4):
    """Pinned host->device and device->host copies at once, one stream per
    direction (the traffic of an end-to-end step): their summed bandwidth,
    measured with CUDA events."""
    dev_a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dev_b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    host_a = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    host_b = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    up, down = torch.cuda.Stream(), torch.cuda.Stream()

    def run(n):
        cur = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        up.wait_event(e0)
        down.wait_event(e0)
        with torch.cuda.stream(up):
            for _ in range(n):
                dev_a.copy_(host_a, non_blocking=True)
        with torch.cuda.stream(down):
            for _ in range(n):
                host_b.copy_(dev_b, non_blocking=True)
        cur.wait_stream(up)
        cur.wait_stream(down)
        e1.record(cur)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    run(1)
    gbs = 2 * reps * nbytes / (run(reps) * 1e-3) / 1e9
    del dev_a, dev_b, host_a, host_b
    return gbs


def e2e_link_fields(e2e, bidir_gbs):
    """The end-to-end step's link traffic (its upload plus its image) per
    second, against pinned copies in both directions at once."""
    moved = (e2e["h2d_bytes_per_step"] + e2e["d2h_bytes_per_step"]) / (e2e["ms_per_step"] * 1e-3) / 1e9
    return {"link_gbs": round(moved, 2), "link_bidir_measured_gbs": round(bidir_gbs, 2),
            "frac_of_link_bidir": round(moved / bidir_gbs, 4),
            "link_what": "upload + image bytes per step over ms_per_step, against pinned "
                         "host->device and device->host copies running at once"}


def run_oversub(args):
    """Section 4.4's synthetic benchmark: two vectors of 2^32 fp32 (32 GiB) in
    managed memory on a GPU that holds half of them.  A device-memory ballast
    leaves the application 16 GiB of HBM (plus the library's working set, 2
    GiB of scratch), so the footprint really oversubscribes the device:
    vector a sits on the device, vector b in host memory.  Each step
    rewrites 2 % of the pages of both (a seeded scatter) and checkpoints
    (null sink).  Two forms of the same steps:
    - in place (managed_in_place=1, the value): b's pages are hashed and
      gathered where they are, over the link, and stay there;
    - the driver's default, run first: a set without managed_in_place takes
      one full and two incremental checkpoints, and the capture's reads
      fault b's pages in wherever the driver's policy moves them (the
      paper's data-migration cost)."""
    import torch
    import paper_1808_00117_b300 as crum
    from paper_1808_00117_b300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    crum.load()
    dev = torch.device("cuda", local)
    wl = W.workload("oversub")
    S, n_pages = wl.total_bytes, wl.n_pages
    steps, warmup = args.steps, max(args.warmup, 3)
    link_d2h, link_h2d = link_d2h_peak(torch), link_h2d_peak(torch)
    # the managed ranges start in host memory: the driver keeps device memory
    # it once gave to managed pages, so the ballast must come before any of
    # them reaches the device
    a_buf, b_buf = (W.managed_empty(n, local, where="host") for n in wl.sizes)
    pages_a = W.pages_of(wl.sizes[0])
    k = int(round(wl.dirty_frac * n_pages))
    staging = 2 * (int(1.5 * k) + 1) * W.PAGE
    scatter = {}
    for t in range(1, warmup + steps + 8):
        chosen = W.choose_step(wl, t, n_pages)
        gen = np.random.default_rng(wl.seed * 31 + t)
        masks = torch.as_tensor(gen.integers(1, 2**62, size=chosen.size, dtype=np.int64) | 1, device=dev)
        in_a = chosen < pages_a
        scatter[t] = [(buf.view(torch.int64), torch.as_tensor(pages * (W.PAGE // 8), device=dev), masks[sel])
                      for buf, pages, sel in ((a_buf, chosen[in_a], torch.as_tensor(in_a, device=dev)),
                                              (b_buf, chosen[~in_a] - pages_a,
                                               torch.as_tensor(~in_a, device=dev)))]

    def app_update(t):
        for w64, idx, m in scatter[t]:
            w64[idx] = w64[idx] ^ m

    sets = {}
    for form, flag in (("in_place", 1), ("default", 0)):
        st = crum.CheckpointSet(device=local, staging_bytes=staging, sink=crum.SINK_NULL,
                                managed_in_place=flag)
        for b in (a_buf, b_buf):
            st.register(b.data_ptr(), b.numel())
        sets[form] = st
    probe_out = torch.empty(W.pages_of(1 << 30), dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    hbm_left = wl.meta["device_holds_bytes"] + (2 << 30)
    ballast = torch.empty(max(0, free - hbm_left), dtype=torch.uint8, device=dev)
    ballast_bytes = ballast.numel()
    for i, b in enumerate((a_buf, b_buf)):
        W.fill_(b, wl.seed * 7919 + i + 1000 * rank, wl.kind)
    W.managed_prefetch(b_buf.data_ptr(), b_buf.numel(), "host", local)
    W.managed_prefetch(a_buf.data_ptr(), a_buf.numel(), "device", local)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def b_read_gbs():
        # a device pass over b's first GiB: HBM rate if its pages moved in,
        # the link's if they are still in host memory
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        crum.hash_pages(b_buf.data_ptr(), 1 << 30, probe_out.data_ptr(), sh)
        e1.record(stream)
        torch.cuda.synchronize()
        return round((1 << 30) / (e0.elapsed_time(e1) * 1e-3) / 1e9, 1)

    # the driver's default placement policy first, before any advice was
    # ever given for these ranges: full + 2 incremental checkpoints
    s0 = sets["default"]
    d_infos = []
    for j, flags in enumerate((crum.FULL, crum.INCR, crum.INCR)):
        if j:
            app_update(warmup + steps + 2 + j)
        im = s0.checkpoint(sh, flags)
        im.wait()
        d_infos.append(im.info())
        im.release()
    b_after_default = b_read_gbs()
    s0.destroy()
    # back to the application's placement for the in-place form
    W.managed_prefetch(b_buf.data_ptr(), b_buf.numel(), "host", local)
    W.managed_prefetch(a_buf.data_ptr(), a_buf.numel(), "device", local)
    torch.cuda.synchronize()
    # in place
    s = sets["in_place"]
    full = s.checkpoint(sh, crum.FULL)
    full.wait()
    full_info = full.info()
    full.release()
    for t in range(1, warmup + 1):
        app_update(t)
        s.checkpoint(sh).wait()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    launches0 = crum.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark("t0")
    e0.record(stream)
    timed = []
    for t in range(warmup + 1, warmup + steps + 1):
        app_update(t)
        timed.append(s.checkpoint(sh))
    for img in timed:
        img.wait(crum.WAIT_DRAINED)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    barrier(dist)
    launches = crum.kernel_launches() - launches0
    clk = clocks.stop()
    for img in timed:
        img.wait()
    infos = [img.info() for img in timed]
    for img in timed:
        img.release()
    b_after_in_place = b_read_gbs()
    s.destroy()
    total_ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)
    cap_ms = [i["t_hash_ms"] + i["t_compact_ms"] for i in infos]
    hash_ms = [i["t_hash_ms"] for i in infos]
    mean_cap = max_over_ranks(dist, statistics.mean(cap_ms), dev)
    mean_hash = max_over_ranks(dist, statistics.mean(hash_ms), dev)
    host_bytes = wl.sizes[1]
    achieved = host_bytes / (mean_hash * 1e-3) / 1e9
    drain_gbs = statistics.mean(i["image_bytes"] / (i["t_drain_ms"] * 1e-3) / 1e9 for i in infos)
    assert all(i["host_pages"] == W.pages_of(wl.sizes[1]) for i in infos)

    del ballast
    line = {
        "metric": METRIC, "value": round(world * S / (mean_cap * 1e-3) / 1e9, 2), "unit": UNIT,
        "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": round(total_ms / steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.name, "footprint_bytes": S, "kind": wl.kind,
                   "vectors": "2 x 2^32 fp32 in managed memory",
                   "placement": "a on the device, b in host memory; a device-memory ballast, "
                                "allocated before any managed page reached the device, leaves "
                                "the managed ranges 18 GiB of HBM (a's 16 GiB + 2 GiB)",
                   "ballast_bytes": int(ballast_bytes),
                   "dirty_pages_per_step": int(statistics.mean(i["n_dirty"] for i in infos)),
                   "sink": "null", "staging_bytes": staging, "managed_in_place": 1},
        "roofline": {"kernel": "k_hash_dirty", "bound": "host link",
                     "what": "b's 16 GiB read in place over the link (a's 16 GiB from HBM beside it)",
                     "achieved": round(achieved, 1), "peak": round(link_h2d, 2), "unit": "GB/s",
                     "frac": round(achieved / link_h2d, 4), "traffic": None,
                     "peak_source": "pinned host->device copy measured in this run"},
        "capture": {"ms_mean": round(statistics.mean(cap_ms), 3),
                    "hash_ms_mean": round(statistics.mean(hash_ms), 3)},
        "drain": {"gbs": round(drain_gbs, 2), "link_measured_gbs": round(link_d2h, 2),
                  "frac_measured": round(drain_gbs / link_d2h, 4)},
        "latency_ms": {"captured_p50": pct([i["t_captured_ms"] for i in infos], 50),
                       "captured_p99": pct([i["t_captured_ms"] for i in infos], 99),
                       "drained_p50": pct([i["t_drained_ms"] for i in infos], 50),
                       "drained_p99": pct([i["t_drained_ms"] for i in infos], 99)},
        "full_checkpoint": {"captured_ms": round(full_info["t_captured_ms"], 1),
                            "drained_ms": round(full_info["t_drained_ms"], 1),
                            "hash_ms": round(full_info["t_hash_ms"], 1)},
        "driver_default": {"what": "a set without managed_in_place, run first (no advice ever given "
                                   "for these ranges): full + 2 incremental",
                           "captured_ms": [round(i["t_captured_ms"], 1) for i in d_infos],
                           "hash_ms": [round(i["t_hash_ms"], 1) for i in d_infos],
                           "drained_ms": [round(i["t_drained_ms"], 1) for i in d_infos]},
        "b_read_gbs_after": {"in_place": b_after_in_place, "driver_default": b_after_default,
                             "link_h2d_gbs": round(link_h2d, 2)},
        "clocks": clk, "gpu_launches": int(launches),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    import paper_1808_00117_b300 as crum
    from paper_1808_00117_b300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    crum.load()
    dev = torch.device("cuda", local)
    wl = bench_workload(args)
    S = wl.total_bytes
    n_pages = wl.n_pages
    k_dirty = int(round(wl.dirty_frac * n_pages))
    incr_image = 64 + 16 * len(wl.sizes) + 16 * k_dirty + 8 + k_dirty * W.PAGE
    full_image = 64 + 16 * len(wl.sizes) + 16 * n_pages + 8 + n_pages * W.PAGE
    steps, warmup = args.steps, max(args.warmup, 3)

    link_peak = link_d2h_peak(torch)
    bufs = []
    memory = app_memory(args, wl)
    for i, n in enumerate(wl.sizes):
        b = app_alloc(torch, memory, n, dev)
        W.fill_(b, wl.seed * 7919 + i + 1000 * rank, wl.kind)
        bufs.append(b)
    torch.cuda.synchronize()
    staging = 2 * ((n_pages + 1) * W.PAGE)  # two halves that each hold every page
    pool = full_image + (warmup + steps + 2) * incr_image
    fixed = [int(x) for x in args.mapping.split(",")] if args.mapping else None
    sink_dir = None
    if args.sink == "file":
        sink_dir = tempfile.mkdtemp(prefix="crum_sink_")
    s = crum.CheckpointSet(device=local, staging_bytes=staging, host_pool_bytes=pool,
                           use_graph=int(args.graph),
                           hash_mapping=fixed[0] if fixed else -1,
                           gather_mapping=fixed[1] if fixed else -1,
                           sink=crum.SINK_FILE if sink_dir else crum.SINK_MEMORY,
                           sink_dir=sink_dir, fsync=int(bool(sink_dir)), compress=int(args.compress))
    for b in bufs:
        s.register(b.data_ptr(), b.numel())
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    full = s.checkpoint(sh, crum.FULL)
    full.wait()
    if fixed:
        tune = {"hash_mapping": fixed[0], "gather_mapping": fixed[1], "hash_ms": [], "gather_ms": []}
    else:
        tune = s.autotune()  # untimed: picks the hash and gather thread mappings
    chain = [full]
    offsets = np.cumsum([0] + [W.pages_of(n) for n in wl.sizes])

    # the application's page choices are drawn up front (host-side numpy),
    # so the timed steps hold only the application's update kernels
    choices = {}
    for step in range(1, warmup + steps + 6):  # + the verify-mode and rollback steps
        pages = W.choose_step(wl, step, n_pages)
        per = []
        for i, b in enumerate(bufs):
            loc = pages[(pages >= offsets[i]) & (pages < offsets[i + 1])] - offsets[i]
            n_full = b.numel() // W.PAGE
            per.append((torch.as_tensor(loc[loc < n_full], device=dev), bool((loc == n_full).any())))
        choices[step] = per

    def app_update(step):
        for i, b in enumerate(bufs):
            full_pages, tail = choices[step][i]
            W.mutate_pages_(b, full_pages, wl.seed + 17 * step + i, has_tail=tail)

    for step in range(warmup):
        app_update(step + 1)
        chain.append(s.checkpoint(sh))
    for img in chain:
        img.wait()

    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    launches0 = crum.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark("t0")
    e0.record(stream)
    timed = []
    t_loop0 = time.perf_counter()
    for step in range(steps):
        app_update(warmup + 1 + step)
        timed.append(s.checkpoint(sh))
    for img in timed:
        img.wait(crum.WAIT_DRAINED)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    barrier(dist)
    launches = crum.kernel_launches() - launches0
    clk = clocks.stop()
    for img in timed:
        img.wait()
    writer_s = time.perf_counter() - t_loop0
    chain.extend(timed)
    total_ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)

    infos = [img.info() for img in timed]
    cap_ms = [i["t_hash_ms"] + i["t_compact_ms"] for i in infos]
    hash_ms = [i["t_hash_ms"] for i in infos]
    drain_ms = [i["t_drain_ms"] for i in infos]
    drained_bytes = [i["image_bytes"] for i in infos]
    mean_cap = max_over_ranks(dist, statistics.mean(cap_ms), dev)
    mean_hash = max_over_ranks(dist, statistics.mean(hash_ms), dev)
    value = world * S / (mean_cap * 1e-3) / 1e9
    peaks = measured_peaks()
    hash_bytes = S + 16 * n_pages  # read every page, read + write each committed hash
    achieved = hash_bytes / (mean_hash * 1e-3) / 1e9
    drain_gbs = statistics.mean(b / (t * 1e-3) / 1e9 for b, t in zip(drained_bytes, drain_ms))

    # restore of the chain end (full image + every incremental) onto
    # garbage, in both forms: merged (the set's automatic choice for this
    # chain: every page once, from its newest image) and replay (every
    # image in turn, through a second set on the same allocations)
    def timed_restore(target):
        for b in bufs:
            W.fill_(b, 4242, "u32")
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        target.restore(chain[-1], sh)
        r1.record(stream)
        torch.cuda.synchronize()
        return r0.elapsed_time(r1)

    replay_set = crum.CheckpointSet(device=local, staging_bytes=2 << 30,
                                    restore_mode=crum.RESTORE_REPLAY)
    for b in bufs:
        replay_set.register(b.data_ptr(), b.numel())
    replay_ms = timed_restore(replay_set)
    replay_set.destroy()
    restore_ms = timed_restore(s)  # leaves the set's memory at the chain end
    restore_bytes = sum(img.info()["n_dirty"] for img in chain) * W.PAGE
    restore_images = len(chain)
    # rollback: one more application update, then a delta restore of the
    # chain end, which copies only the pages that now differ
    delta_set = crum.CheckpointSet(device=local, staging_bytes=2 * W.PAGE,
                                   restore_mode=crum.RESTORE_DELTA)
    for b in bufs:
        delta_set.register(b.data_ptr(), b.numel())
    app_update(warmup + steps + 5)
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    delta_set.restore(chain[-1], sh)
    d1.record(stream)
    torch.cuda.synchronize()
    rollback = {"ms": round(d0.elapsed_time(d1), 3), "pages_copied": delta_set.restore_pages(),
                "what": "delta restore of the chain end after one more application update "
                        "(5 % of pages rewritten): pages whose hash differs are copied"}
    delta_set.destroy()

    # plain form P0 (Section 3.4): synchronize, then copy every allocation
    # whole to pinned host memory (through one 1 GiB pinned buffer, so that
    # ranks sharing a host do not each pin the whole footprint; the copies
    # are the same link-bound bytes)
    host_plain = torch.empty(min(S, 1 << 30), dtype=torch.uint8, pin_memory=True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    p0.record(stream)
    for b in bufs:
        for off in range(0, b.numel(), host_plain.numel()):
            m = min(host_plain.numel(), b.numel() - off)
            host_plain[:m].copy_(b[off:off + m], non_blocking=True)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    del host_plain

    for img in chain:
        img.release()
    chain = []
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, crum, W, s, bufs, wl, steps, sh, stream, warmup + steps + 1, dist, dev, world)

    # verify mode (exact byte compare against a device shadow of the last
    # checkpointed contents): the hash pass then reads every page and its
    # shadow; a few untimed-setup steps, device-timed like the main loop
    verify = None
    if not args.no_verify:
        # null sink: only tables and the bounce region are pinned
        vs = crum.CheckpointSet(device=local, staging_bytes=staging, verify=1, sink=crum.SINK_NULL)
        for b in bufs:
            vs.register(b.data_ptr(), b.numel())
        vs.checkpoint(sh, crum.FULL | crum.VERIFY).wait()
        vinfo = []
        for j in range(4):
            app_update(warmup + steps + 1 + j)  # steps the timed loop did not use
            im = vs.checkpoint(sh, crum.VERIFY)
            im.wait()
            vinfo.append(im.info())
            im.release()
        vinfo = vinfo[1:]
        vms = statistics.mean(i["t_hash_ms"] for i in vinfo)
        verify = {"hash_ms": round(vms, 4), "read_bytes": 2 * S,
                  "gbs": round(2 * S / (vms * 1e-3) / 1e9, 1),
                  "frac": round(2 * S / (vms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                  "collisions": int(sum(i["collisions"] for i in vinfo)),
                  "what": "verify-mode hash pass: every page and its shadow read once"}
        vs.destroy()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # a single-GPU run's baseline
        cb = oracle_cpu_baseline(wl, args.cpu_sample_mib, 3, 1, bool(args.compress))
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "all_cores")}

    traffic = traffic_from_profile("k_hash_dirty", wl.name)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": round(total_ms / steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": wl.name, "footprint_bytes": S, "allocations": len(wl.sizes),
                   "n_pages": n_pages, "dirty_pages_per_step": k_dirty,
                   "memory": MEMORY_DESC[memory], "kind": wl.kind,
                   "images": "compressed (byte-plane dictionary code)" if args.compress else "plain",
                   "staging_bytes": staging, "parallelism": f"replica per GPU x{world}",
                   "l2": f"inputs ({S / 2**30:g} GiB) larger than L2 (126 MB); no flush",
                   "value_def": "footprint bytes / capture-kernel device time (hash+scan+gather)",
                   "capture_launch": "cuda graph" if args.graph else "one launch per op",
                   "hash_mapping": tune["hash_mapping"], "gather_mapping": tune["gather_mapping"],
                   "autotune_hash_ms": [round(x, 4) for x in tune["hash_ms"]],
                   "autotune_gather_ms": [round(x, 4) for x in tune["gather_ms"]]},
        "roofline": {"kernel": "k_hash_dirty", "bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                     "peak_source": peaks["source"], "bytes_per_launch": hash_bytes,
                     "ms_per_launch": round(statistics.mean(hash_ms), 4)},
        "capture": {"ms_mean": round(statistics.mean(cap_ms), 4),
                    "hash_ms_mean": round(statistics.mean(hash_ms), 4),
                    "frac_of_hbm": round(value / world / peaks["hbm_gbs"], 4),
                    **({"encode_ms_mean": round(statistics.mean(i["t_encode_ms"] for i in infos), 4),
                        "encode_what": "compressed images: device time from captured to code and "
                                       "trailer written (size, offsets, encode, checksum)"}
                       if args.compress else {})},
        "drain": {"gbs": round(drain_gbs, 2), "link_measured_gbs": round(link_peak, 2),
                  "frac_measured": round(drain_gbs / link_peak, 4),
                  "effective_gbs": round(statistics.mean(
                      raw_image_bytes(i) / (i["t_drain_ms"] * 1e-3) / 1e9 for i in infos), 2),
                  "link_nominal_gbs": NOMINAL_LINK_GBS,
                  "frac_nominal": round(drain_gbs / NOMINAL_LINK_GBS, 4),
                  "bytes_per_step": int(statistics.mean(drained_bytes))},
        "latency_ms": {"captured_p50": pct([i["t_captured_ms"] for i in infos], 50),
                       "captured_p99": pct([i["t_captured_ms"] for i in infos], 99),
                       "drained_p50": pct([i["t_drained_ms"] for i in infos], 50),
                       "drained_p99": pct([i["t_drained_ms"] for i in infos], 99),
                       "persisted_p50": pct([i["t_persisted_ms"] for i in infos], 50),
                       "persisted_p99": pct([i["t_persisted_ms"] for i in infos], 99),
                       "n": len(infos)},
        "restore": {"images": restore_images, "form": "merged", "ms": round(restore_ms, 3),
                    "chain_payload_bytes": restore_bytes, "link_bytes": S,
                    "chain_gbs": round(restore_bytes / (restore_ms * 1e-3) / 1e9, 2),
                    "link_gbs": round(S / (restore_ms * 1e-3) / 1e9, 2),
                    "replay_ms": round(replay_ms, 3), "rollback": rollback,
                    "replay_link_gbs": round(restore_bytes / (replay_ms * 1e-3) / 1e9, 2),
                    "what": "chain end restored onto garbage; chain_gbs = the chain's payload "
                            "bytes / ms (what replaying the chain would move)"},
        "plain_p0": {"ms": round(plain_ms, 3), "gbs": round(S / (plain_ms * 1e-3) / 1e9, 2),
                     "what": "synchronize + full device->host copy of the footprint"},
        "verify": verify,
        "writer": {"sink": args.sink, "fsync": args.sink == "file",
                   "persisted_gbs": round(sum(drained_bytes) / writer_s / 1e9, 2),
                   "what": "image bytes of the timed steps / host time from the first "
                           "submit until every image is persisted"},
        "whole_step": {"gbs": round(world * S / (total_ms / steps * 1e-3) / 1e9, 2),
                       "what": "footprint bytes / wall-clock ms per step; each step also drains "
                               "its dirty pages over the host link"},
        "clocks": clk,
        "gpu_launches": int(launches),
        "cpu_baseline": cpu,
        "e2e": e2e,
    }
    for img in chain:
        img.release()
    s.destroy()
    if sink_dir:
        import shutil
        shutil.rmtree(sink_dir, ignore_errors=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_e2e(torch, crum, W, s, bufs, wl, steps, sh, stream, step0, dist, dev, world):
    """Public API end to end: each step copies the application's new page
    contents host->device from pinned memory, checkpoints, and reads the
    image back (PERSISTED: its bytes crossed device->host).  Two forms, each
    step holding its own uploads and its own image drain:
    - pipelined (the value): step k+1's upload is issued before waiting for
      image k-1 (two images in flight), on a copy stream into one of two
      landing buffers, so it overlaps step k's capture and shares the
      full-duplex link with the previous drains, as an application that
      keeps running while its checkpoints drain would;
    - serial: each step waits for its image before the next upload.
    Images are released once persisted, so the pinned pool is reused."""
    n_pages = wl.n_pages
    k = int(round(wl.dirty_frac * n_pages))
    gen = torch.Generator(device="cpu")
    gen.manual_seed(wl.seed + 99)
    new = torch.randint(0, 256, (k, W.PAGE), dtype=torch.uint8, generator=gen).pin_memory()
    n_full = bufs[0].numel() // W.PAGE
    pages_view = bufs[0][:n_full * W.PAGE].view(n_full, W.PAGE)
    # two landing buffers on a copy stream: step k+1's host->device copy may
    # run while step k's capture and drain do; only the scatter into the
    # application's memory is ordered after the capture (on the app stream)
    landing = [torch.empty((k, W.PAGE), dtype=torch.uint8, device=dev) for _ in range(2)]
    scattered = [None, None]  # app-stream event after the scatter that read landing[j]
    copy_stream = torch.cuda.Stream(device=dev)
    plan = []
    for step in range(2 * steps + 4):
        p = W.choose_step(wl, step0 + step, n_pages)
        plan.append(torch.as_tensor(p[p < n_full], device=dev))
    turn = [0]

    def upload(idx, ev=None):
        # the application's new page contents: one pinned host->device copy
        # of the step's pages, then a device scatter into place
        m, j = int(idx.numel()), turn[0]
        turn[0] ^= 1
        with torch.cuda.stream(copy_stream):
            if scattered[j] is not None:
                copy_stream.wait_event(scattered[j])
            if ev is not None:
                ev[0].record(copy_stream)
            landing[j][:m].copy_(new[:m], non_blocking=True)
            if ev is not None:
                ev[1].record(copy_stream)
            landed = torch.cuda.Event()
            landed.record(copy_stream)
        stream.wait_event(landed)
        pages_view.index_copy_(0, idx, landing[j][:m])
        scattered[j] = torch.cuda.Event()
        scattered[j].record(stream)
        return m * W.PAGE

    def finish(im, infos):
        im.wait()
        infos.append(im.info())
        im.release()

    def fresh_chain():
        # untimed: a fresh full image starts a new chain, so the previous
        # chain (kept alive by its newest image) is freed and its pinned
        # memory reused
        im = s.checkpoint(sh, crum.FULL)
        im.wait()
        im.release()

    def timed(first_step, pipelined):
        h2d, infos, ev = [], [], []
        for warm in range(2):
            upload(plan[first_step + warm])
            finish(s.checkpoint(sh), [])
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pending = []
        for step in range(steps):
            u = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            h2d.append(upload(plan[first_step + 2 + step], u))
            ev.append(u)
            pending.append(s.checkpoint(sh))
            # pipelined: two images stay in flight, so the next upload is
            # queued while the one before it still runs and the copy engine
            # moving host-to-device never idles; serial: none
            while len(pending) > (2 if pipelined else 0):
                finish(pending.pop(0), infos)
        while pending:
            finish(pending.pop(0), infos)
        torch.cuda.synchronize()
        dt = max_over_ranks(dist, time.perf_counter() - t0, dev)
        return dt, h2d, infos, statistics.mean(a.elapsed_time(b) for a, b in ev)

    fresh_chain()
    dt, h2d, infos, up_ms = timed(0, True)
    fresh_chain()
    dt_s, _, infos_s, up_ms_s = timed(steps + 2, False)
    per = lambda x: round(world * wl.total_bytes * steps / x / 1e9, 2)
    out = {"value": per(dt), "unit": UNIT,
            "h2d_bytes_per_step": int(statistics.mean(h2d)),
            "d2h_bytes_per_step": int(statistics.mean(i["image_bytes"] for i in infos)),
            "ms_per_step": round(dt * 1e3 / steps, 3),
            "what": "pinned H2D of the step's new pages (copy stream, two landing buffers) + device "
                    "scatter + crum_checkpoint + image read back (PERSISTED); two images in flight, "
                    "step k+1's upload overlaps image k's capture and the drains",
            "submit_to_persisted_ms": round(statistics.mean(i["t_persisted_ms"] for i in infos), 3),
            "upload_ms": round(up_ms, 3),
            "serial": {"value": per(dt_s), "ms_per_step": round(dt_s * 1e3 / steps, 3),
                       "upload_ms": round(up_ms_s, 3),
                       "submit_to_persisted_ms":
                           round(statistics.mean(i["t_persisted_ms"] for i in infos_s), 3),
                       "what": "each step waits for its image before the next upload"}}
    out.update(e2e_link_fields(out, link_bidir_peak(torch)))
    return out


def run_e2e_carved(torch, crum, W, bufs, big, wl, page_byte, page_valid, steps, sh, stream,
                   step0, dist, dev, world, local, tune, staging):
    """Public API end to end on a footprint carved out of one tensor into
    many allocations (the large workload): each step copies the new contents
    of the step's pages host->device from pinned memory (one copy), scatters
    them into place on the device (the allocations' pages start on 4 KiB
    boundaries, so the scatter moves 4 KiB blocks; a tail page moves only
    its valid blocks), checkpoints through a memory-sink set, and reads the
    image back (PERSISTED: its bytes are in host memory).

    Host memory bounds the form: the chain base is drained without keeping
    its payload (a 140 GiB full image does not fit the host beside its
    incrementals), and each form runs at most 8 steps, since an incremental
    image holds its parent and so every image of a form stays pinned until
    the form ends.  Pipelined (the value: two images in flight, step k+1's
    upload on a copy stream overlapping image k's capture and the drains)
    and serial (each step waits for its image) as in ``run_e2e``."""
    BLK = 4096
    assert all(n % BLK == 0 for n in wl.sizes)
    n_pages = wl.n_pages
    k_est = int(round(wl.dirty_frac * n_pages)) + 64
    img_est = 64 + 16 * len(wl.sizes) + (16 + W.PAGE) * k_est + 8
    # a form's images stay pinned until it ends: fit them in this rank's
    # share of host memory (8 steps on one GPU of this node)
    e_steps = min(steps, 8, host_budget_bytes() // img_est - 4)
    if e_steps < 2:
        return None
    blocks = big.view(torch.int64).view(-1, BLK // 8)
    plan = []
    for step in range(2 * e_steps + 4):
        p = W.choose_step(wl, step0 + step, n_pages)
        starts = page_byte[p] // BLK
        counts = page_valid[p] // BLK
        off = np.repeat(np.cumsum(counts) - counts, counts)
        idx = np.repeat(starts, counts) + (np.arange(int(counts.sum())) - off)
        plan.append((torch.as_tensor(idx, device=dev), int(p.size)))
    rows = max(int(ix.numel()) for ix, _ in plan)
    k_max = max(k for _, k in plan)
    gen = torch.Generator(device="cpu")
    gen.manual_seed(wl.seed + 99)
    new = torch.randint(-2**62, 2**62, (rows, BLK // 8), dtype=torch.int64, generator=gen).pin_memory()
    landing = [torch.empty((rows, BLK // 8), dtype=torch.int64, device=dev) for _ in range(2)]
    scattered = [None, None]
    copy_stream = torch.cuda.Stream(device=dev)
    img_bytes = 64 + 16 * len(wl.sizes) + 16 * k_max + 8 + k_max * W.PAGE
    es = crum.CheckpointSet(device=local, staging_bytes=staging, sink=crum.SINK_MEMORY,
                            host_pool_bytes=(e_steps + 4) * img_bytes + (64 << 20),
                            hash_mapping=tune["hash_mapping"], gather_mapping=tune["gather_mapping"])
    for b in bufs:
        es.register(b.data_ptr(), b.numel())
    turn = [0]

    def copy_in(j_plan, ev=None):
        # the step's new page contents: one pinned host->device copy into a
        # landing buffer, on the copy stream (once the scatter that last read
        # that buffer is done)
        idx, _ = plan[j_plan]
        m, j = int(idx.numel()), turn[0]
        turn[0] ^= 1
        with torch.cuda.stream(copy_stream):
            if scattered[j] is not None:
                copy_stream.wait_event(scattered[j])
            if ev is not None:
                ev[0].record(copy_stream)
            landing[j][:m].copy_(new[:m], non_blocking=True)
            if ev is not None:
                ev[1].record(copy_stream)
            landed = torch.cuda.Event()
            landed.record(copy_stream)
        return idx, m, j, landed

    def scatter(c):
        # on the application's stream: into place, 4 KiB blocks
        idx, m, j, landed = c
        stream.wait_event(landed)
        blocks.index_copy_(0, idx, landing[j][:m])
        scattered[j] = torch.cuda.Event()
        scattered[j].record(stream)
        return m * BLK

    def upload(j_plan, ev=None):
        return scatter(copy_in(j_plan, ev))

    def finish(im, infos):
        im.wait()
        infos.append(im.info())
        im.release()

    def fresh_chain():
        # untimed: a new chain base whose payload crosses the link but is
        # not kept, so the previous chain is freed and its pinned memory reused
        im = es.checkpoint(sh, crum.FULL | crum.NO_PAYLOAD)
        im.wait()
        im.release()

    def timed(first, pipelined):
        # pipelined: the copy of step k+1's pages is issued before step k's
        # checkpoint call, which returns only once the hash pass is done when
        # staging cannot hold every page of the set, so the link carries that
        # copy while step k is captured and step k-1 drains; two images stay
        # in flight.  Serial: each step waits for its image first.
        h2d, infos, ev = [], [], []
        for warm in range(2):
            upload(first + warm)
            finish(es.checkpoint(sh), [])
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pending = []
        pair = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        nxt = None
        for step in range(e_steps):
            if nxt is None:
                u = pair()
                cur = (copy_in(first + 2 + step, u), u)
            else:
                cur = nxt
            nxt = None
            if pipelined and step + 1 < e_steps:
                u = pair()
                nxt = (copy_in(first + 3 + step, u), u)
            ev.append(cur[1])
            h2d.append(scatter(cur[0]))
            pending.append(es.checkpoint(sh))
            while len(pending) > (2 if pipelined else 0):
                finish(pending.pop(0), infos)
        while pending:
            finish(pending.pop(0), infos)
        torch.cuda.synchronize()
        dt = max_over_ranks(dist, time.perf_counter() - t0, dev)
        return dt, h2d, infos, statistics.mean(a.elapsed_time(b) for a, b in ev)

    fresh_chain()
    dt, h2d, infos, up_ms = timed(0, True)
    fresh_chain()
    dt_s, _, infos_s, up_ms_s = timed(e_steps + 2, False)
    es.destroy()
    del landing, new
    per = lambda x: round(world * wl.total_bytes * e_steps / x / 1e9, 2)
    out = {"value": per(dt), "unit": UNIT,
            "h2d_bytes_per_step": int(statistics.mean(h2d)),
            "d2h_bytes_per_step": int(statistics.mean(i["image_bytes"] for i in infos)),
            "ms_per_step": round(dt * 1e3 / e_steps, 3), "steps": e_steps,
            "what": "pinned H2D of the step's new page contents (copy stream, two landing "
                    "buffers; step k+1's copy issued before step k's checkpoint call) + device "
                    "scatter of 4 KiB blocks + crum_checkpoint (memory sink) + image read back "
                    "(PERSISTED); two images in flight",
            "submit_to_persisted_ms": round(statistics.mean(i["t_persisted_ms"] for i in infos), 3),
            "upload_ms": round(up_ms, 3),
            "serial": {"value": per(dt_s), "ms_per_step": round(dt_s * 1e3 / e_steps, 3),
                       "upload_ms": round(up_ms_s, 3),
                       "persisted_p50_ms": pct([i["t_persisted_ms"] for i in infos_s], 50),
                       "persisted_p99_ms": pct([i["t_persisted_ms"] for i in infos_s], 99),
                       "what": "each step waits for its image before the next upload"}}
    out.update(e2e_link_fields(out, link_bidir_peak(torch)))
    return out


def stencil_dirty_pages(wl, plans):
    """Global pages a stencil step rewrites (pages overlapping its planes)."""
    from paper_1808_00117_b300 import workloads as W
    plane = 8 * W.STENCIL_NX * W.STENCIL_NY
    out, g0 = [], 0
    for n, plan in zip(wl.sizes, plans):
        if plan is not None:
            _, z0, L = plan
            lo, hi = z0 * plane // W.PAGE, ((z0 + L) * plane - 1) // W.PAGE
            out.extend(range(g0 + lo, g0 + hi + 1))
        g0 += W.pages_of(n)
    return out


def run_batched(args):
    """Many uneven allocations (the stencil-shaped footprint): one batched
    capture launch over the flattened page list, against the plain form P1
    (one set, hence one hash/scan/gather launch sequence, per allocation).
    Null sink: images cross the host link and are then dropped, so host
    memory stays bounded over many steps."""
    import torch
    import paper_1808_00117_b300 as crum
    from paper_1808_00117_b300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    crum.load()
    dev = torch.device("cuda", local)
    wl = bench_workload(args)
    S, n_pages = wl.total_bytes, wl.n_pages
    steps, warmup = args.steps, max(args.warmup, 3)
    link_peak = link_d2h_peak(torch)
    stencil = wl.dirty_mode == "stencil"
    bufs = []
    memory = app_memory(args, wl)
    if stencil:
        for i, n in enumerate(wl.sizes):
            b = app_alloc(torch, memory, n, dev)
            W.fill_(b, wl.seed * 7919 + i + 1000 * rank, wl.kind)
            bufs.append(b)
        plans = {t: [W.stencil_plan(n, wl.dirty_frac, wl.seed * 1000 + 7 * t + i)
                     for i, n in enumerate(wl.sizes)] for t in range(1, warmup + steps + 8)}
        dirty = {t: len(stencil_dirty_pages(wl, plans[t])) for t in plans}

        def app_update(t):
            for b, plan in zip(bufs, plans[t]):
                W.stencil_step_(b, plan)
    else:
        # one device tensor carved into the allocations (offsets are 4 KiB
        # multiples); the application's update is one seeded scatter that
        # xors a nonzero mask into the first word of every chosen page
        big = app_alloc(torch, memory, S, dev)
        W.fill_(big, wl.seed + 1000 * rank, wl.kind)
        offs = np.cumsum([0] + list(wl.sizes))
        bufs = [big[int(offs[i]):int(offs[i + 1])] for i in range(len(wl.sizes))]
        page_byte = np.concatenate([offs[i] + np.arange(W.pages_of(n), dtype=np.int64) * W.PAGE
                                    for i, n in enumerate(wl.sizes)])
        big64 = big.view(torch.int64)
        scatter, dirty = {}, {}
        # the timed and warm-up steps, then the restore leg's updates
        for t in list(range(1, warmup + steps + 8)) + list(range(warmup + steps + 40, warmup + steps + 48)):
            chosen = W.choose_step(wl, t, n_pages)
            gen = np.random.default_rng(wl.seed * 31 + t)
            masks = gen.integers(1, 2**62, size=chosen.size, dtype=np.int64) | 1
            scatter[t] = (torch.as_tensor(page_byte[chosen] // 8, device=dev),
                          torch.as_tensor(masks, device=dev))
            dirty[t] = int(chosen.size)

        def app_update(t):
            idx, m = scatter[t]
            big64[idx] = big64[idx] ^ m

    torch.cuda.synchronize()
    if stencil:
        staging = 2 * (n_pages + 1) * W.PAGE  # both halves hold every page
    else:
        staging = 2 * (int(1.5 * max(dirty.values())) + 1) * W.PAGE  # halves hold a step's pages
    # null sink: an image keeps only its header and tables in host memory
    # (the payload crosses the link into the 64 MiB bounce region)
    tables = 64 + 16 * len(wl.sizes) + 16 * n_pages + 8
    fixed = [int(x) for x in args.mapping.split(",")] if args.mapping else None
    s = crum.CheckpointSet(device=local, staging_bytes=staging, sink=crum.SINK_NULL,
                           host_pool_bytes=4 * ((tables + 4095) // 4096 * 4096) + (64 << 20),
                           compress=int(args.compress), managed_in_place=int(args.managed_in_place),
                           hash_mapping=fixed[0] if fixed else -1,
                           gather_mapping=fixed[1] if fixed else -1, use_graph=int(args.graph))
    for b in bufs:
        s.register(b.data_ptr(), b.numel())
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    s.checkpoint(sh, crum.FULL).wait()
    if fixed:
        tune = {"hash_mapping": fixed[0], "gather_mapping": fixed[1], "hash_ms": [], "gather_ms": []}
    else:
        tune = s.autotune()  # untimed: picks the hash and gather thread mappings
    for t in range(1, warmup + 1):
        app_update(t)
        s.checkpoint(sh).wait()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    launches0 = crum.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark("t0")
    e0.record(stream)
    timed = []
    for t in range(warmup + 1, warmup + steps + 1):
        app_update(t)
        timed.append(s.checkpoint(sh))
    for img in timed:
        img.wait(crum.WAIT_DRAINED)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    barrier(dist)
    launches = crum.kernel_launches() - launches0
    clk = clocks.stop()
    for img in timed:
        img.wait()
    infos = [img.info() for img in timed]
    for img in timed:
        img.release()
    total_ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)
    cap_ms = [i["t_hash_ms"] + i["t_compact_ms"] for i in infos]
    hash_ms = [i["t_hash_ms"] for i in infos]
    mean_cap = max_over_ranks(dist, statistics.mean(cap_ms), dev)
    mean_hash = max_over_ranks(dist, statistics.mean(hash_ms), dev)
    peaks = measured_peaks()
    hash_bytes = S + 16 * n_pages
    achieved = hash_bytes / (mean_hash * 1e-3) / 1e9
    drain_gbs = statistics.mean(i["image_bytes"] / (i["t_drain_ms"] * 1e-3) / 1e9 for i in infos)
    assert [i["n_dirty"] for i in infos] == [dirty[t] for t in range(warmup + 1, warmup + steps + 1)]

    # batched vs plain P1 at equal bytes: application-stream time from the
    # submit until every dirty page is captured, staging idle beforehand
    p1_steps = min(3, steps)
    p1_what = "one set (hash, scan and gather launches) per allocation"
    p1_sets = []
    if not stencil:
        # thousands of one-allocation sets would need two host threads each;
        # compare the hash pass alone: one launch over the flattened page list
        # against one launch per allocation, same thread mapping (1)
        p1_what = "hash pass only: one launch per allocation vs one batched launch (mapping 1)"
        out = torch.empty(n_pages, dtype=torch.int64, device=dev)
        plain_ms_hash = []
        for j in range(p1_steps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            g = 0
            for b in bufs:
                crum.hash_pages(b.data_ptr(), b.numel(), out[g:].data_ptr(), sh)
                g += W.pages_of(b.numel())
            a1.record(stream)
            torch.cuda.synchronize()
            plain_ms_hash.append(a0.elapsed_time(a1))
        # the set's own batched hash over the flattened list, same mapping
        batched_ms_hash = [tune["hash_ms"][1] if tune["hash_ms"] else statistics.mean(hash_ms)] * p1_steps
        del out
    for b in (bufs if stencil else []):
        n_b = W.pages_of(b.numel())
        ps = crum.CheckpointSet(device=local, staging_bytes=2 * (n_b + 1) * W.PAGE,
                                sink=crum.SINK_NULL, hash_mapping=tune["hash_mapping"],
                                gather_mapping=tune["gather_mapping"])
        ps.register(b.data_ptr(), b.numel())
        ps.checkpoint(sh, crum.FULL).wait()
        p1_sets.append(ps)
    batched_ms, plain_ms = [], []
    if not stencil:
        batched_ms, plain_ms = batched_ms_hash, plain_ms_hash
    base_t = warmup + steps + 1
    for j in range(p1_steps if stencil else 0):
        app_update(base_t + j)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        imgs = [ps.checkpoint(sh) for ps in p1_sets]
        a1.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(a0.elapsed_time(a1))
        for im in imgs:
            im.wait()
            im.release()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        im = s.checkpoint(sh)
        b1.record(stream)
        torch.cuda.synchronize()
        batched_ms.append(b0.elapsed_time(b1))
        im.wait()
        im.release()
    for ps in p1_sets:
        ps.destroy()

    # one checkpoint at a time with the pipeline empty (the application
    # otherwise idle): the latency of a checkpoint taken every few seconds,
    # beside the timed steps' back-to-back latency
    iso = []
    for t in range(warmup + steps + 4, warmup + steps + 7):
        app_update(t)
        torch.cuda.synchronize()
        im = s.checkpoint(sh)
        im.wait()
        iso.append(im.info())
        im.release()
    isolated = {"n": len(iso),
                "captured_ms": [round(i["t_captured_ms"], 2) for i in iso],
                "drained_ms": [round(i["t_drained_ms"], 2) for i in iso],
                "what": "one checkpoint at a time, staging and link idle at the submit"}

    extra = {}
    if not stencil:
        extra = large_legs(args, torch, crum, W, s, bufs, big, wl, page_byte, offs, steps, warmup,
                           sh, stream, dist, dev, world, local, tune, staging, rank, app_update)
    line = {
        "metric": METRIC, "value": round(world * S / (mean_cap * 1e-3) / 1e9, 2), "unit": UNIT,
        "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": round(total_ms / steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.name, "footprint_bytes": S, "allocations": len(wl.sizes),
                   "n_pages": n_pages, "dirty_pages_per_step": int(statistics.mean(i["n_dirty"] for i in infos)),
                   "sink": "null", "staging_bytes": staging, "memory": MEMORY_DESC[memory],
                   "kind": wl.kind, "managed_in_place": int(args.managed_in_place),
                   "images": "compressed (byte-plane dictionary code)" if args.compress else "plain",
                   "hash_mapping": tune["hash_mapping"], "gather_mapping": tune["gather_mapping"],
                   "autotune_hash_ms": [round(x, 4) for x in tune["hash_ms"]],
                   "autotune_gather_ms": [round(x, 4) for x in tune["gather_ms"]]},
        "roofline": {"kernel": "k_hash_dirty", "bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": None,
                     "peak_source": peaks["source"]},
        "capture": {"ms_mean": round(statistics.mean(cap_ms), 4),
                    "hash_ms_mean": round(statistics.mean(hash_ms), 4),
                    **({"encode_ms_mean": round(statistics.mean(i["t_encode_ms"] for i in infos), 4)}
                       if args.compress else {})},
        "drain": {"gbs": round(drain_gbs, 2), "link_measured_gbs": round(link_peak, 2),
                  "frac_measured": round(drain_gbs / link_peak, 4),
                  "effective_gbs": round(statistics.mean(
                      raw_image_bytes(i) / (i["t_drain_ms"] * 1e-3) / 1e9 for i in infos), 2)},
        "latency_ms": {"captured_p50": pct([i["t_captured_ms"] for i in infos], 50),
                       "captured_p99": pct([i["t_captured_ms"] for i in infos], 99),
                       "drained_p50": pct([i["t_drained_ms"] for i in infos], 50),
                       "drained_p99": pct([i["t_drained_ms"] for i in infos], 99),
                       "isolated": isolated},
        "batched_vs_plain_p1": {"steps": p1_steps, "what": p1_what,
                                "batched_capture_ms": [round(x, 3) for x in batched_ms],
                                "plain_p1_capture_ms": [round(x, 3) for x in plain_ms],
                                "speedup": round(statistics.mean(plain_ms) / statistics.mean(batched_ms), 3)},
        "clocks": clk, "gpu_launches": int(launches),
    }
    if extra:
        line["roofline"]["traffic"] = extra.pop("traffic")
        line["roofline"]["bytes_per_launch"] = S + 16 * n_pages
        line["roofline"]["ms_per_launch"] = round(statistics.mean(hash_ms), 4)
        line["config"]["l2"] = (f"inputs ({S / 2**30:g} GiB) larger than L2 (126 MB); no flush")
        line["config"]["value_def"] = ("footprint bytes / capture-kernel device time "
                                       "(hash+scan+gather)")
        line["config"]["capture_launch"] = (
            ("cuda graph" if args.graph else "one launch per op") if staging // 2 // W.PAGE >= n_pages
            else "chunked: staging halves hold 1.5x a step's dirty pages, so the call waits for "
                 "the dirty count after the hash pass and launches the gather itself")
        line["config"]["parallelism"] = f"replica per GPU x{world}"
        line["capture"]["frac_of_hbm"] = round(S / (statistics.mean(cap_ms) * 1e-3) / 1e9
                                               / peaks["hbm_gbs"], 4)
        line["drain"].update({"link_nominal_gbs": NOMINAL_LINK_GBS,
                              "frac_nominal": round(drain_gbs / NOMINAL_LINK_GBS, 4),
                              "bytes_per_step": int(statistics.mean(i["image_bytes"] for i in infos))})
        line["latency_ms"]["n"] = len(infos)
        line["latency_ms"]["persisted_p50"] = extra["e2e"]["serial"]["persisted_p50_ms"] \
            if extra.get("e2e") else None
        line["latency_ms"]["persisted_p99"] = extra["e2e"]["serial"]["persisted_p99_ms"] \
            if extra.get("e2e") else None
        line["latency_ms"]["what"] = ("captured and drained: the timed steps (null sink: each image "
                                      "crosses the link into a bounce region); persisted: the e2e "
                                      "leg's serial steps (memory sink, image bytes in host memory); "
                                      "back-to-back steps are drain-bound, so a capture waits for the "
                                      "staging half whose drain is in flight")
        drain_ms = statistics.mean(i["t_drain_ms"] for i in infos)
        line["whole_step"] = {"gbs": round(world * S / (total_ms / steps * 1e-3) / 1e9, 2),
                              "drain_ms": round(drain_ms, 3),
                              "what": "footprint bytes / wall-clock ms per step; the step is bound by "
                                      "its drain (drain_ms of each step's image over the host link)"}
        line.update(extra)
    else:
        s.destroy()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def restore_prefix(torch, crum, W, bufs, big, wl, sh, stream, dev, local, tune, staging, app_update,
                   t0, limit=40 << 30, n_incr=4):
    """Restore of a chain of the large workload's shape.  The whole footprint
    cannot be restored here: its full image (140 GiB) does not fit in host
    memory beside its incrementals.  The allocations in registration order
    up to `limit` bytes (a prefix of the footprint) form their own set with a
    memory sink: a full image, `n_incr` incrementals of the application's 2 %
    updates, the prefix scribbled, the chain end restored (merged: every
    page once, from its newest image, read over the link by the kernel),
    and the prefix compared whole on the device with its state at the
    chain end."""
    k, tot = 0, 0
    while k < len(wl.sizes) and tot + wl.sizes[k] <= limit:
        tot += wl.sizes[k]
        k += 1
    pages = sum(W.pages_of(n) for n in wl.sizes[:k])
    full_img = 64 + 16 * k + 16 * pages + 8 + pages * W.PAGE
    incr = int(1.2 * wl.dirty_frac * pages) + 64
    rs = crum.CheckpointSet(device=local, staging_bytes=staging, sink=crum.SINK_MEMORY,
                            host_pool_bytes=full_img + (n_incr + 1) * (64 + 16 * k + (16 + W.PAGE) * incr + 8),
                            hash_mapping=tune["hash_mapping"], gather_mapping=tune["gather_mapping"],
                            restore_mode=crum.RESTORE_MERGED)
    for b in bufs[:k]:
        rs.register(b.data_ptr(), b.numel())
    chain = [rs.checkpoint(sh, crum.FULL)]
    chain[0].wait()
    for t in range(n_incr):
        app_update(t0 + t)
        chain.append(rs.checkpoint(sh))
    for im in chain:
        im.wait()
    payload = sum(im.info()["n_dirty"] for im in chain) * W.PAGE
    torch.cuda.synchronize()
    expect = big[:tot].clone()
    W.fill_(big[:tot], 4242, "u32")
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    rs.restore(chain[-1], sh)
    r1.record(stream)
    torch.cuda.synchronize()
    ms = r0.elapsed_time(r1)
    equal = bool(torch.equal(big[:tot], expect))
    del expect
    for im in chain:
        im.release()
    rs.destroy()
    if not equal:
        print("restored prefix differs from its state at the chain end", file=sys.stderr)
    return {"form": "merged", "ms": round(ms, 3), "images": len(chain), "allocations": k,
            "footprint_bytes": tot, "chain_payload_bytes": payload,
            "link_gbs": round(tot / (ms * 1e-3) / 1e9, 2), "restored_equal": equal,
            "what": f"the first {k} allocations of the workload ({tot / 2**30:.1f} GiB, the most the "
                    "host holds as a kept full image beside its incrementals): full + "
                    f"{n_incr} incrementals of the application's updates, prefix scribbled, chain "
                    "end restored and compared whole on the device"}


def large_legs(args, torch, crum, W, s, bufs, big, wl, page_byte, offs, steps, warmup, sh, stream,
               dist, dev, world, local, tune, staging, rank, app_update):
    """The large workload's other measurements, after its timed steps: the
    public API end to end, the plain form P0, the CPU oracle, and what is
    not measured at this footprint and why."""
    S = wl.total_bytes
    s.destroy()  # frees the timed set's staging before the e2e set takes its own
    torch.cuda.synchronize()
    out = {}
    page_valid = np.concatenate([np.minimum(W.PAGE, n - np.arange(W.pages_of(n), dtype=np.int64) * W.PAGE)
                                 for n in wl.sizes])
    out["e2e"] = None if args.no_e2e else run_e2e_carved(
        torch, crum, W, bufs, big, wl, page_byte, page_valid, steps, sh, stream,
        warmup + steps + 8, dist, dev, world, local, tune, staging)

    # plain form P0 (Section 3.4): synchronize, then copy the footprint whole
    # to pinned host memory, through one 1 GiB pinned buffer
    host_plain = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    p0.record(stream)
    for off in range(0, S, host_plain.numel()):
        m = min(host_plain.numel(), S - off)
        host_plain[:m].copy_(big[off:off + m], non_blocking=True)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    del host_plain
    out["plain_p0"] = {"ms": round(plain_ms, 3), "gbs": round(S / (plain_ms * 1e-3) / 1e9, 2),
                       "what": "synchronize + full device->host copy of the footprint"}
    # the prefix's full image and incrementals must fit this rank's share of
    # host memory (40 GiB on one GPU of this node)
    prefix = min(40 << 30, int(host_budget_bytes() / 1.2))
    out["restore"] = None if args.no_restore or prefix < (1 << 30) else restore_prefix(
        torch, crum, W, bufs, big, wl, sh, stream, dev, local, tune, staging, app_update,
        warmup + steps + 40, limit=prefix)
    out["verify"] = {"measured": False,
                     "why": "verify mode keeps a device shadow of the footprint: 140 GiB beside "
                            "140 GiB does not fit in HBM (measured on uint32_8g)"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_cpu_baseline(wl, args.cpu_sample_mib, 3, 1, bool(args.compress))
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "all_cores")}
    out["cpu_baseline"] = cpu
    name = wl.name if not wl.meta.get("resized_gib") else None
    out["traffic"] = traffic_from_profile("k_hash_dirty", name) if name else None
    return out


def run_serving(args):
    """Checkpoint/restore requests from 32 simulated clients through
    crum_server: footprints log-uniform 1 MiB..4 GiB (int32/fp32/fp64 in
    turn), 80 % checkpoints (every 4th of a client full, so chains stay
    short) and 20 % restores of the client's newest chain, each checkpoint
    and each restore preceded by the client rewriting U[1 %, 50 %] of its
    pages (a restore rolls them back: delta restores copy the pages that
    differ).  For each of 3 seeds (request mix and arrival times):
    the sequential form of the server (one request on the device at a time)
    saturated gives its service rate mu; then Poisson arrivals at 0.8 mu
    through the sequential form, through continuous batching (8 slots,
    16 GiB staging budget; two lane settings) and through the plain form
    (one request at a time: synchronize, then copy the client's whole
    footprint device->host for a checkpoint or host->device for a restore,
    the paper's naive capture, Section 3.4).  Then batching and the plain
    form saturated.  One driver thread per client replays that client's
    requests at their arrival times."""
    import threading
    import torch
    import paper_1808_00117_b300 as crum
    from paper_1808_00117_b300 import workloads as W

    torch.cuda.set_device(0)
    crum.load()
    n_clients, n_req = 32, args.requests
    sizes = W.workload("serving").sizes
    kinds = ["i32", "fp32", "fp64"]
    budget = 16 << 30

    class C:
        pass

    clients = []
    for i, n in enumerate(sizes):
        c = C()
        c.size, c.pages = n, W.pages_of(n)
        c.buf = torch.empty(n, dtype=torch.uint8, device="cuda")
        W.fill_(c.buf, 7000 + i, {"i32": "u32", "fp32": "fp32", "fp64": "fp64"}[kinds[i % 3]])
        c.stream = torch.cuda.Stream()
        clients.append(c)
    torch.cuda.synchronize()

    # sets (and their pinned pools) are reused by every run.  A client's
    # pool holds its chain: a full image, up to three incrementals of at most
    # half its pages (every fourth checkpoint is full) and the next full
    # image while the old chain is still referenced, 3.5 footprints at most;
    # a pool that had to grow in the middle of the run would pin host memory
    # (hundreds of ms for a GB, holding the driver's locks) while every other
    # client waits
    for c in clients:
        c.set = crum.CheckpointSet(external_staging=1, host_pool_bytes=4 * c.size + (16 << 20),
                                   restore_mode=crum.RESTORE_DELTA)
        c.set.register(c.buf.data_ptr(), c.size)

    def requests(seed):
        rng = np.random.default_rng(0x5EED + 3 + 1000 * seed)
        return (rng.integers(0, n_clients, size=n_req), rng.random(n_req) < 0.2,
                rng.uniform(0.01, 0.50, size=n_req))

    def arrivals(seed, rate_hz):
        gaps = (np.random.default_rng(17 + seed).exponential(1.0 / rate_hz, size=n_req)
                if rate_hz else np.zeros(n_req))
        return np.cumsum(gaps)

    def summary(label, lat_all, lat_ck, lat_rs, wall_s, bytes_ck, extra=None):
        out = {"label": label, "completed": len(lat_all),
               "throughput_req_s": round(len(lat_all) / wall_s, 2),
               "checkpointed_gbs": round(bytes_ck / wall_s / 1e9, 2),
               "p50_ms": round(pct(lat_all, 50), 3), "p99_ms": round(pct(lat_all, 99), 3),
               "p50_ckpt_ms": round(pct(lat_ck, 50), 3), "p99_ckpt_ms": round(pct(lat_ck, 99), 3),
               "p50_restore_ms": round(pct(lat_rs, 50), 3), "p99_restore_ms": round(pct(lat_rs, 99), 3)}
        out.update(extra or {})
        return out

    def run(seed, max_inflight, rate_hz, label, max_ckpt=0, max_rest=0, serial=0, order=0):
        req_client, req_restore, req_frac = requests(seed)
        srv = crum.Server(staging_budget=budget, max_inflight=max_inflight,
                          max_checkpoints=max_ckpt, max_restores=max_rest, serialize_drains=serial,
                          order=order)
        for c in clients:
            c.cid = srv.add_client(c.set, c.stream.cuda_stream)
            c.n_ckpt = 0
        # warm-up: every client's first request is a full checkpoint
        for c in clients:
            srv.wait(srv.submit(c.cid, crum.REQ_CHECKPOINT_FULL))
            c.n_ckpt = 1
        srv.reset_stats()
        arr = arrivals(seed, rate_hz)
        per_client = [[] for _ in clients]
        for r in range(n_req):
            per_client[req_client[r]].append(r)
        t0 = time.perf_counter() + 0.05
        ids = [None] * n_req

        def drive(ci):
            c = clients[ci]
            last = None
            for r in per_client[ci]:
                delay = t0 + arr[r] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                if last is not None:  # the client's consistency rule
                    srv.wait(last[0], crum.WAIT_CAPTURED if last[1] != crum.REQ_RESTORE else crum.WAIT_PERSISTED)
                # the request's share of rewritten pages: a checkpoint
                # captures them, a restore rolls them back
                k = max(1, int(round(req_frac[r] * c.pages)))
                pages = W.choose_uniform(int(r) * 31 + ci, c.pages, k)
                with torch.cuda.stream(c.stream):
                    W.mutate_pages_(c.buf, pages, int(r))
                if req_restore[r]:
                    kind = crum.REQ_RESTORE
                else:
                    kind = crum.REQ_CHECKPOINT_FULL if c.n_ckpt % 4 == 0 else crum.REQ_CHECKPOINT
                    c.n_ckpt += 1
                ids[r] = srv.submit(c.cid, kind)
                last = (ids[r], kind)

        threads = [threading.Thread(target=drive, args=(ci,)) for ci in range(n_clients)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        st = srv.drain()
        wall_s = st["wall_ms"] * 1e-3
        out = {"label": label, "seed": seed, "max_inflight": max_inflight,
               "max_checkpoints": max_ckpt, "max_restores": max_rest, "serialize_drains": serial,
               "order": "size-first" if order else "arrival",
               "arrival_rate_hz": None if not rate_hz else round(rate_hz, 2),
               "completed": st["completed"], "failed": st["failed"],
               "throughput_req_s": round(st["completed"] / wall_s, 2),
               "checkpointed_gbs": round(st["bytes_checkpointed"] / wall_s / 1e9, 2),
               "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
               "p50_ckpt_ms": round(st["p50_ckpt_ms"], 3), "p99_ckpt_ms": round(st["p99_ckpt_ms"], 3),
               "p50_restore_ms": round(st["p50_restore_ms"], 3),
               "p99_restore_ms": round(st["p99_restore_ms"], 3),
               "peak_inflight": st["peak_inflight"], "peak_staging_bytes": st["peak_staging"]}
        srv.destroy()
        return out

    # the plain form's host images: one pinned buffer per client
    plain_host = [torch.empty(c.size, dtype=torch.uint8, pin_memory=True) for c in clients]

    def run_plain(seed, rate_hz, label):
        """One request at a time in arrival order: the client's rewrite, a
        device synchronize, then the whole footprint copied across the link
        (device->host for a checkpoint, host->device for a restore)."""
        req_client, req_restore, req_frac = requests(seed)
        for c, h in zip(clients, plain_host):  # warm-up: every client's first image
            h.copy_(c.buf)
        torch.cuda.synchronize()
        arr = arrivals(seed, rate_hz)
        t0 = time.perf_counter() + 0.05
        lat_all, lat_ck, lat_rs, bytes_ck = [], [], [], 0
        for r in range(n_req):
            ci = int(req_client[r])
            c, h = clients[ci], plain_host[ci]
            delay = t0 + arr[r] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            k = max(1, int(round(req_frac[r] * c.pages)))
            pages = W.choose_uniform(int(r) * 31 + ci, c.pages, k)
            with torch.cuda.stream(c.stream):
                W.mutate_pages_(c.buf, pages, int(r))
            torch.cuda.synchronize()
            if req_restore[r]:
                c.buf.copy_(h)
            else:
                h.copy_(c.buf)
                bytes_ck += c.size
            torch.cuda.synchronize()
            ms = (time.perf_counter() - (t0 + arr[r])) * 1e3
            lat_all.append(ms)
            (lat_rs if req_restore[r] else lat_ck).append(ms)
        wall_s = time.perf_counter() - t0 - (arr[0] if rate_hz else 0.0)
        return summary(label, lat_all, lat_ck, lat_rs, wall_s, bytes_ck,
                       {"seed": seed, "arrival_rate_hz": None if not rate_hz else round(rate_hz, 2),
                        "what": "plain form: synchronize + whole-footprint copy per request"})

    launches0 = crum.kernel_launches()
    runs, per_seed = [], []
    # batched: 8 slots, two checkpoints and one restore on the device at once,
    # admitted smallest expected transfer first (with aging); beside it the
    # same lanes in arrival order with serialized drains
    for seed in range(3):
        seq_sat = run(seed, 1, 0, "sequential, saturated", serial=-1)
        lam = 0.8 * seq_sat["throughput_req_s"]
        seq = run(seed, 1, lam, "sequential, Poisson 0.8 mu", serial=-1)
        bat = run(seed, 8, lam, "batched 2/1 size-first, Poisson 0.8 mu", 2, 1, -1, 1)
        bat_s = run(seed, 8, lam, "batched 2/1 arrival order, serialized drains, Poisson 0.8 mu", 2, 1, 1)
        plain = run_plain(seed, lam, "plain, Poisson 0.8 mu")
        runs += [seq_sat, seq, bat, bat_s, plain]
        per_seed.append({"seed": seed, "lambda_req_s": round(lam, 2),
                         "p50_ms": {"plain": plain["p50_ms"], "sequential": seq["p50_ms"],
                                    "batched": bat["p50_ms"], "batched_arrival_order": bat_s["p50_ms"]},
                         "p99_ms": {"plain": plain["p99_ms"], "sequential": seq["p99_ms"],
                                    "batched": bat["p99_ms"], "batched_arrival_order": bat_s["p99_ms"]},
                         "batched_p99_below_plain": bat["p99_ms"] < plain["p99_ms"],
                         "batched_p99_below_sequential": bat["p99_ms"] < seq["p99_ms"]})
    bat_sat = run(0, 8, 0, "batched 2/1 size-first, saturated", 2, 1, -1, 1)
    alt_sat = run(0, 8, 0, "batched 2/1 arrival order, serialized drains, saturated", 2, 1, 1)
    plain_sat = run_plain(0, 0, "plain, saturated")
    seq_sat0 = runs[0]
    runs += [bat_sat, alt_sat, plain_sat]
    line = {
        "metric": METRIC, "value": bat_sat["checkpointed_gbs"], "unit": UNIT, "n_gpus": 1,
        "steps": n_req, "warmup": n_clients, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "serving", "clients": n_clients, "requests": n_req,
                   "footprint_bytes": int(sum(sizes)), "staging_budget": budget,
                   "restore_share": 0.2, "dirty": "U[1%,50%] per request", "seeds": 3,
                   "value_def": "footprint bytes checkpointed per second, batched saturated"},
        "per_seed": per_seed,
        "runs": runs,
        "saturated_throughput_req_s": {"plain": plain_sat["throughput_req_s"],
                                       "sequential": seq_sat0["throughput_req_s"],
                                       "batched": bat_sat["throughput_req_s"],
                                       "batched_arrival_order": alt_sat["throughput_req_s"]},
        "gpu_launches": int(crum.kernel_launches() - launches0),
    }
    for c in clients:
        c.set.destroy()
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload in ("stencil", "large"):
        return run_batched(args)
    if args.workload == "oversub":
        return run_oversub(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
