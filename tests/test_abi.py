"""The C-ABI library loads and exports every symbol include/crum.h declares
(no GPU needed; no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1808_00117_b300 as crum

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "crum.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(crum_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["crum_set_create", "crum_register", "crum_checkpoint", "crum_image_wait",
              "crum_restore", "crum_image_save", "crum_image_load", "crum_image_release"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = crum.load()
    for n in declared_functions():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", crum.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (crum_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_signatures_cover_the_header():
    assert set(declared_functions()) == set(crum.SIGNATURES)


def test_build_targets_sm_103a_only():
    from paper_1808_00117_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_calls():
    assert crum.version().startswith("crum-b300")
    c = crum.config()
    assert c.staging_bytes == 1 << 30 and c.chunk_bytes == 64 << 20 and c.sink == crum.SINK_MEMORY
    assert crum.load().crum_last_error() == b""


def test_argument_errors_need_no_device():
    lib = crum.load()
    assert lib.crum_register(None, None, 0, None) == crum.EINVAL
    assert lib.crum_checkpoint(None, None, 0, None) == crum.EINVAL
    assert lib.crum_image_wait(None, 1, 0) == crum.EINVAL
    assert lib.crum_hash_pages(None, 0, None, None) == crum.EINVAL
    assert b"null" in lib.crum_last_error()
    cfg = crum.config(staging_bytes=1000)
    h = ctypes.c_void_p()
    assert lib.crum_set_create(ctypes.byref(cfg), ctypes.byref(h)) == crum.EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and
    field offsets (a C program compiled from include/crum.h prints them)."""
    structs = {"crum_config": crum.Config, "crum_image_info": crum.ImageInfo,
               "crum_server_config": crum.ServerConfig, "crum_request_info": crum.RequestInfo,
               "crum_server_stats": crum.ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "crum.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, f"{cname}.{f}"


def test_mapping_counts_match_the_header():
    src = open(os.path.join(ROOT, "include", "crum.h")).read()
    h = int(re.search(r"#define CRUM_NUM_HASH_MAPPINGS (\d+)", src).group(1))
    g = int(re.search(r"#define CRUM_NUM_GATHER_MAPPINGS (\d+)", src).group(1))
    assert (crum.NUM_HASH_MAPPINGS, crum.NUM_GATHER_MAPPINGS) == (h, g)
