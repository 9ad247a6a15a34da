"""Restart in a new process (Section 3.4): one process checkpoints a chain
to image files and exits; this process loads the files into a set of its
own over fresh allocations of the same sizes and restores the chain end.
The memory equals the first process's final state and the oracle's restore
of the same files, for plain and compressed images."""
from __future__ import annotations

import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W

from helpers import host_copies, make_set, stream_handle, torch

pytestmark = pytest.mark.gpu
P = W.PAGE
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W
sink, compress = sys.argv[1], int(sys.argv[2])
sizes = [int(x) for x in sys.argv[3].split(",")]
bufs = []
for i, n in enumerate(sizes):
    b = torch.empty(n, dtype=torch.uint8, device="cuda")
    W.fill_(b, 4100 + i, "fp32")
    bufs.append(b)
torch.cuda.synchronize()
s = crum.CheckpointSet(sink=crum.SINK_FILE, sink_dir=sink, compress=compress, fsync=1)
for b in bufs:
    s.register(b.data_ptr(), b.numel())
sh = torch.cuda.current_stream().cuda_stream
for step in range(3):
    if step:
        for i, (b, n) in enumerate(zip(bufs, sizes)):
            pages = np.arange(step - 1, W.pages_of(n), 3)
            if pages.size:
                W.mutate_pages_(b, pages, 4200 + 10 * step + i)
        torch.cuda.synchronize()
    img = s.checkpoint(sh)
    img.wait()
    img.release()
for i, b in enumerate(bufs):
    b.cpu().numpy().tofile(f"{sink}/final_{i}.bin")
s.destroy()
print("done")
"""


@pytest.fixture(autouse=True)
def _cuda():
    t = torch()
    if not t.cuda.is_available():
        pytest.skip("needs a CUDA device")
    crum.load()
    yield
    t.cuda.synchronize()


@pytest.mark.parametrize("compress", [0, 1])
def test_restart_from_files_in_a_new_process(tmp_path, compress):
    sizes = [9 * P + 24, 4 * P, 100]
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    out = subprocess.run([sys.executable, "-c", CHILD, str(tmp_path), str(compress),
                          ",".join(map(str, sizes))], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0 and "done" in out.stdout, out.stderr
    final = [np.fromfile(tmp_path / f"final_{i}.bin", dtype=np.uint8) for i in range(len(sizes))]
    files = sorted((f for f in tmp_path.iterdir() if f.suffix == ".img"),
                   key=lambda f: int(f.stem.rsplit("_", 1)[1]))
    assert len(files) == 3
    data = [f.read_bytes() for f in files]
    for d in data:
        assert oracle.check_image(d) == oracle.OK
        assert oracle.image_version(d) == (2 if compress else 1)
    # the oracle's restart from the same files onto zeroed host memory
    host = [np.zeros(n, dtype=np.uint8) for n in sizes]
    assert oracle.OracleSet(sizes).restore(data, host) == oracle.OK
    assert all(np.array_equal(h, f) for h, f in zip(host, final))
    # this process's restart through the C ABI onto scribbled device memory
    t = torch()
    bufs = [t.full((n,), 0xC3, dtype=t.uint8, device="cuda") for n in sizes]
    r = make_set(bufs)
    chain = []
    for f in files:
        chain.append(r.load_image(str(f), chain[-1] if chain else None))
    r.restore(chain[-1], stream_handle())
    t.cuda.synchronize()
    assert all(np.array_equal(g, f) for g, f in zip(host_copies(bufs), final))
    for c in chain:
        c.release()
    r.destroy()
