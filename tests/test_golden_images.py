"""Images pinned by stored digests (tests/golden/image_digests.txt, written
from the oracle by tests/golden/make_image_digests.py): the oracle must keep
producing them, and the CUDA path must produce the same bytes."""
from __future__ import annotations

import hashlib
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location(
    "make_image_digests", os.path.join(HERE, "golden", "make_image_digests.py"))
G = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(G)


def stored():
    out = {}
    for line in open(os.path.join(HERE, "golden", "image_digests.txt")):
        if line.startswith("#") or not line.strip():
            continue
        case, k, sha, trailer, n = line.split()
        out.setdefault(case, []).append((sha, int(trailer, 16), int(n)))
    return out


@pytest.mark.parametrize("case", sorted(G.CASES))
def test_oracle_reproduces_stored_images(case):
    assert G.digests(case) == stored()[case]


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(G.CASES))
def test_cuda_path_produces_stored_images(case):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1808_00117_b300 as crum
    sizes, host, steps = G.inputs(case)
    dev = [torch.from_numpy(h.copy()).cuda() for h in host]
    torch.cuda.synchronize()
    s = crum.CheckpointSet(compress=int(G.CASES[case][3]))
    for d in dev:
        s.register(d.data_ptr(), d.numel())
    sh = torch.cuda.current_stream().cuda_stream
    got = []
    for k in range(len(steps) + 1):
        if k:
            for h, d, (chosen, masks) in zip(host, dev, steps[k - 1]):
                G.rewrite(h, chosen, masks)
                d.copy_(torch.from_numpy(h))
            torch.cuda.synchronize()
        img = s.checkpoint(sh)
        img.wait()
        b = img.to_bytes()
        got.append((hashlib.sha256(b).hexdigest(), int(np.frombuffer(b[-8:], dtype=np.uint64)[0]), len(b)))
        img.release()
    s.destroy()
    assert got == stored()[case]
