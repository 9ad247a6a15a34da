"""Compressed images (crum_config.compress): the CUDA path's version-2
images equal the oracle's byte for byte, for float pages (which shrink),
random words (stored as is) and ragged tails; every restore form brings the
chain back; files round-trip; the checksum of a payload that is not kept
still matches."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W

from helpers import device_buffers, first_diff, host_copies, make_set, mutate, stream_handle, torch

pytestmark = pytest.mark.gpu
P = W.PAGE
SIZES = [1, 4096 + 8, P - 8, P, 3 * P + 40, 21 * P + 4104]


@pytest.fixture(autouse=True)
def _cuda():
    t = torch()
    if not t.cuda.is_available():
        pytest.skip("needs a CUDA device")
    crum.load()
    yield
    t.cuda.synchronize()


def _ckpt(s, flags=crum.INCR):
    img = s.checkpoint(stream_handle(), flags)
    img.wait()
    return img, img.to_bytes()


@pytest.mark.parametrize("kind", ["fp32", "fp64", "bf16", "u32"])
def test_compressed_images_equal_the_oracle(kind):
    bufs = device_buffers(SIZES, seed=81, kind=kind)
    s = make_set(bufs, compress=1)
    o = oracle.OracleSet(SIZES, compress=True)
    raw = oracle.OracleSet(SIZES)
    for step in range(3):
        if step:
            mutate(bufs, SIZES, 0.4, seed=810 + step)
        img, got = _ckpt(s)
        state = host_copies(bufs)
        exp, *_ = o.checkpoint(state)
        plain, *_ = raw.checkpoint(state)
        assert oracle.image_version(got) == 2
        assert first_diff(got, exp) is None, f"step {step}"
        assert img.info()["image_bytes"] == len(exp)
        assert img.info()["t_encode_ms"] > 0  # the encoding stage was timed
        if kind in ("fp32", "fp64", "bf16") and step == 0:
            assert len(got) < 0.95 * len(plain)
        img.release()
    s.destroy()


def test_compressed_capture_as_one_graph():
    """use_graph: the encoding stage runs as nodes of the capture graph;
    images stay byte-identical, including after a registration change
    rebuilds the graph."""
    bufs = device_buffers(SIZES, seed=93, kind="fp32")
    s = make_set(bufs, compress=1, use_graph=1)
    o = oracle.OracleSet(SIZES, compress=True)
    for step in range(3):
        if step:
            mutate(bufs, SIZES, 0.3, seed=930 + step)
        img, got = _ckpt(s)
        exp, *_ = o.checkpoint(host_copies(bufs))
        assert first_diff(got, exp) is None, f"step {step}"
        assert img.info()["t_encode_ms"] > 0
        img.release()
    extra = device_buffers([5 * P + 16], seed=94, kind="fp32")
    s.register(extra[0].data_ptr(), extra[0].numel())
    sizes = SIZES + [5 * P + 16]
    o.register(5 * P + 16)
    for step in range(2):
        if step:
            mutate(bufs + extra, sizes, 0.3, seed=940 + step)
        img, got = _ckpt(s)
        exp, *_ = o.checkpoint(host_copies(bufs + extra))
        assert first_diff(got, exp) is None, f"after the change, step {step}"
        img.release()
    s.destroy()


@pytest.mark.parametrize("mode", [crum.RESTORE_REPLAY, crum.RESTORE_MERGED, crum.RESTORE_DELTA])
def test_compressed_chain_restores(mode):
    bufs = device_buffers(SIZES, seed=83, kind="fp32")
    s = make_set(bufs, compress=1, restore_mode=mode)
    chain, states = [], []
    for step in range(3):
        if step:
            mutate(bufs, SIZES, 0.3, seed=830 + step)
        img = s.checkpoint(stream_handle())
        img.wait()
        chain.append(img)
        states.append(host_copies(bufs))
    for k in (2, 0, 1):
        for i, b in enumerate(bufs):
            W.fill_(b, 8300 + k + 10 * i, "u32")
        s.restore(chain[k], stream_handle())
        torch().cuda.synchronize()
        assert all(np.array_equal(g, w) for g, w in zip(host_copies(bufs), states[k])), k
        assert s.restore_pages() > 0
    for c in chain:
        c.release()
    s.destroy()


def test_compressed_files_round_trip(tmp_path):
    sizes = [5 * P + 8, 2 * P]
    bufs = device_buffers(sizes, seed=85, kind="fp64")
    s = make_set(bufs, compress=1, sink=crum.SINK_FILE, sink_dir=str(tmp_path))
    states = []
    for step in range(2):
        if step:
            mutate(bufs, sizes, 0.5, seed=850 + step)
        img = s.checkpoint(stream_handle())
        img.wait()
        states.append(host_copies(bufs))
        img.release()
    files = sorted(tmp_path.iterdir(), key=lambda x: int(x.stem.rsplit("_", 1)[1]))
    for f in files:
        assert oracle.check_image(f.read_bytes()) == oracle.OK
    r = make_set(bufs)  # an uncompressed set restores compressed images too
    chain = []
    for f in files:
        chain.append(r.load_image(str(f), chain[-1] if chain else None))
    for i, b in enumerate(bufs):
        W.fill_(b, 8500 + i, "u32")
    r.restore(chain[-1], stream_handle())
    torch().cuda.synchronize()
    assert all(np.array_equal(g, w) for g, w in zip(host_copies(bufs), states[-1]))
    for c in chain:
        c.release()
    r.destroy()
    s.destroy()


def test_compressed_no_payload_and_verify():
    sizes = [300 * P + 24]
    bufs = device_buffers(sizes, seed=87, kind="fp32")
    s = make_set(bufs, compress=1, verify=1)
    o = oracle.OracleSet(sizes, compress=True)
    img = s.checkpoint(stream_handle(), crum.FULL | crum.NO_PAYLOAD)
    img.wait()
    exp, *_ = o.checkpoint(host_copies(bufs))
    assert img.info()["checksum"] == int(np.frombuffer(exp[-8:], dtype=np.uint64)[0])
    assert img.info()["image_bytes"] == len(exp)
    mutate(bufs, sizes, 0.1, seed=871)
    img2 = s.checkpoint(stream_handle(), crum.VERIFY)
    assert img2.wait() == crum.OK
    exp2, *_ = o.checkpoint(host_copies(bufs))
    assert first_diff(img2.to_bytes(), exp2) is None
    s.destroy()


@pytest.mark.parametrize("kind", ["fp32", "u32"])
def test_compressed_chunked_capture_equals_the_oracle(kind):
    # staging of 3 slots per half: the dirty pages are encoded and drained
    # in chunks, each chunk's code placed after the ones before it
    sizes = [20 * P + 40, 7 * P, 8]
    bufs = device_buffers(sizes, seed=91, kind=kind)
    s = make_set(bufs, compress=1, staging_bytes=6 * P)
    o = oracle.OracleSet(sizes, compress=True)
    chain, states = [], []
    for step, frac in enumerate([None, 0.4, 0.0, 0.05]):
        if frac:
            mutate(bufs, sizes, frac, seed=910 + step)
        img, got = _ckpt(s)
        states.append(host_copies(bufs))
        exp, *_ = o.checkpoint(states[-1])
        assert oracle.image_version(got) == 2
        assert first_diff(got, exp) is None, f"step {step}"
        assert img.info()["image_bytes"] == len(exp) and img.info()["t_encode_ms"] > 0
        chain.append(img)
    for mode in (crum.RESTORE_REPLAY, crum.RESTORE_MERGED, crum.RESTORE_DELTA):
        r = make_set(bufs, restore_mode=mode)
        for k in (3, 0, 1):
            for i, b in enumerate(bufs):
                W.fill_(b, 9100 + k + 10 * i, "u32")
            r.restore(chain[k], stream_handle())
            torch().cuda.synchronize()
            assert all(np.array_equal(g, w) for g, w in zip(host_copies(bufs), states[k])), (mode, k)
        r.destroy()
    # a payload that is not kept still crosses the link and is summed
    img = s.checkpoint(stream_handle(), crum.FULL | crum.NO_PAYLOAD)
    img.wait()
    exp, *_ = o.checkpoint(host_copies(bufs), full=True)
    assert img.info()["checksum"] == int(np.frombuffer(exp[-8:], dtype=np.uint64)[0])
    assert img.info()["image_bytes"] == len(exp)
    img.release()
    for c in chain:
        c.release()
    s.destroy()


def test_compression_rejects_external_staging():
    with pytest.raises(crum.CrumError):
        crum.CheckpointSet(compress=1, external_staging=1)


# alphabet sizes per byte plane: each code width b = 0..8 (1 value: b = 0;
# 129 or more: the plane is stored as is)
ALPHABETS = [1, 2, 4, 7, 16, 30, 64, 128, 256]


def alphabet_bytes(n_bytes, seed, shift):
    """Bytes whose page p, byte plane j (byte j of every 64-bit word) draws
    from exactly ALPHABETS[(p + j + shift) % 9] distinct values; the last
    whole page has 256 values in every plane (a slot stored as is) and the
    one before it a single value in every plane (the shortest code)."""
    rng = np.random.default_rng(seed)
    n_pages = W.pages_of(n_bytes)
    out = np.zeros((n_pages, P // 8, 8), dtype=np.uint8)
    whole = n_bytes // P
    for p in range(n_pages):
        for j in range(8):
            k = ALPHABETS[(p + j + shift) % 9]
            if p == whole - 1:
                k = 256
            elif p == whole - 2:
                k = 1
            alph = rng.choice(256, size=k, replace=False).astype(np.uint8)
            vals = alph[rng.integers(0, k, size=P // 8)]
            vals[rng.permutation(P // 8)[:k]] = alph  # every value of the alphabet occurs
            out[p, :, j] = vals
    return out.reshape(-1)[:n_bytes].copy()


@pytest.mark.parametrize("staging_pages", [None, 6])
def test_compressed_every_code_width_equals_the_oracle(staging_pages):
    # every width on every plane, packed words that straddle two threads'
    # runs (odd b), dictionaries of every size, a slot stored as is and a
    # ragged tail; whole images and chunked ones (3 slots per half),
    # trailer included
    t = torch()
    sizes = [20 * P + 4104, 9 * P]
    hosts = [alphabet_bytes(n, seed=4400 + i, shift=i) for i, n in enumerate(sizes)]
    bufs = [t.from_numpy(h).cuda() for h in hosts]
    t.cuda.synchronize()
    cfg = {"compress": 1}
    if staging_pages:
        cfg["staging_bytes"] = staging_pages * P
    s = make_set(bufs, **cfg)
    o = oracle.OracleSet(sizes, compress=True)
    img, got = _ckpt(s, crum.FULL)
    exp, *_ = o.checkpoint(host_copies(bufs), full=True)
    assert first_diff(got, exp) is None
    img.release()
    # rewrite every third page of the first allocation with shifted widths
    new = alphabet_bytes(sizes[0], seed=4500, shift=4)
    for p in range(0, W.pages_of(sizes[0]), 3):
        lo, hi = p * P, min((p + 1) * P, sizes[0])
        bufs[0][lo:hi] = t.from_numpy(new[lo:hi]).cuda()
    t.cuda.synchronize()
    img, got = _ckpt(s)
    exp, *_ = o.checkpoint(host_copies(bufs))
    assert first_diff(got, exp) is None
    assert img.info()["n_dirty"] == len(range(0, W.pages_of(sizes[0]), 3))
    img.release()
    s.destroy()
