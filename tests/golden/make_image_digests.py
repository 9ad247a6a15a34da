"""Writes tests/golden/image_digests.txt: the SHA-256 and trailer of checkpoint
images that the oracle (and only the oracle) produces for small seeded
inputs, so that any later change of the image bytes, by either the oracle or
the CUDA path, fails a test.

Run:  python tests/golden/make_image_digests.py
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
P = 65536

# case name -> (allocation sizes, seed, element kind, compressed form)
CASES = {
    "fp32_ragged": ([3 * P + 100, P - 8, 17, 2 * P], 101, "fp32", False),
    "u64_tails": ([4096, 4096 + 8, P + 24, 5 * P], 202, "u64", False),
    "fp32_ragged_v2": ([3 * P + 100, P - 8, 17, 2 * P], 101, "fp32", True),
    "u64_tails_v2": ([4096, 4096 + 8, P + 24, 5 * P], 202, "u64", True),
}


def inputs(case):
    """Seeded host buffers (numpy only) and, per step, the pages to rewrite."""
    sizes, seed, kind, _ = CASES[case]
    rng = np.random.default_rng(seed)
    bufs = []
    for n in sizes:
        if kind == "fp32":
            words = rng.uniform(-1.0, 1.0, size=(n + 3) // 4).astype(np.float32).view(np.uint8)
        else:
            words = rng.integers(0, 2**64, size=(n + 7) // 8, dtype=np.uint64).view(np.uint8)
        bufs.append(np.ascontiguousarray(words[:n]))
    steps = []
    for step in range(2):
        per = []
        for i, n in enumerate(sizes):
            pages = -(-n // P)
            k = max(1, pages // 3)
            chosen = np.sort(rng.choice(pages, size=k, replace=False))
            masks = rng.integers(1, 256, size=k, dtype=np.uint8)
            per.append((chosen, masks))
        steps.append(per)
    return sizes, bufs, steps


def rewrite(buf, chosen, masks):
    """xor one nonzero byte into every byte of each chosen page (valid bytes)."""
    for p, m in zip(chosen, masks):
        buf[p * P:(p + 1) * P] ^= m


def digests(case):
    sys.path.insert(0, ROOT)
    import oracle
    sizes, bufs, steps = inputs(case)
    o = oracle.OracleSet(sizes, compress=CASES[case][3])
    out = []
    img, *_ = o.checkpoint(bufs)
    out.append(img)
    for per in steps:
        for b, (chosen, masks) in zip(bufs, per):
            rewrite(b, chosen, masks)
        img, *_ = o.checkpoint(bufs)
        out.append(img)
    return [(hashlib.sha256(im).hexdigest(), int(np.frombuffer(im[-8:], dtype=np.uint64)[0]), len(im))
            for im in out]


def main():
    lines = ["# case image sha256 trailer bytes  (written by make_image_digests.py from the oracle)"]
    for case in CASES:
        for k, (sha, trailer, n) in enumerate(digests(case)):
            lines.append(f"{case} {k} {sha} {trailer:016x} {n}")
    with open(os.path.join(HERE, "image_digests.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
