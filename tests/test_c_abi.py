"""The boundary from C: tests/c/abi_roundtrip.c compiled against
include/crum.h and linked with libcrum.so (builds here; runs on a GPU)."""
import os
import subprocess

import pytest

import paper_1808_00117_b300 as crum

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = "/usr/local/cuda"


def _build(tmp_path):
    exe = tmp_path / "abi_roundtrip"
    lib_dir = os.path.dirname(crum.LIB_PATH)
    subprocess.run(["gcc", "-std=c11", "-O2", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c", "abi_roundtrip.c"),
                    "-L", lib_dir, "-lcrum", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                    f"-Wl,-rpath,{lib_dir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}",
                    "-o", str(exe)], check=True)
    return exe


def test_c_program_builds_against_the_header(tmp_path):
    if not os.path.exists(crum.LIB_PATH):
        pytest.skip("library not built")
    assert _build(tmp_path).exists()


@pytest.mark.gpu
def test_c_program_round_trip(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    out = subprocess.run([str(_build(tmp_path))], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "ok"
