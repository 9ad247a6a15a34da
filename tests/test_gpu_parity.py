"""GPU parity: the CUDA library, called through its C ABI, against the CPU
oracle on the same seeded inputs.  Integer and byte work, so the bar is
bit-exact: hashes, dirty sets, page tables, whole images and restored
memory."""
import os

import numpy as np
import pytest

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W

from helpers import (device_buffers, first_diff, host_copies, make_set, mutate, page_offsets,
                     page_table, parse_header, stream_handle, torch)

pytestmark = pytest.mark.gpu

P = 65536
# sizes that exercise full pages, every kind of tail and several tiles
RAGGED = [1, 7, 8, 9, 15, 16, 17, 24, 4096, 4096 + 3, 4096 + 8, P - 8, P, P + 24, 3 * P - 5,
          300 * P + 4104]


@pytest.fixture(autouse=True)
def _cuda():
    t = torch()
    if not t.cuda.is_available():
        pytest.skip("needs a CUDA device")
    crum.load()
    yield
    t.cuda.synchronize()


def test_hash_pages_matches_oracle():
    t = torch()
    bufs = device_buffers(RAGGED, seed=1)
    for b, h in zip(bufs, host_copies(bufs)):
        n = W.pages_of(b.numel())
        out = t.zeros(n, dtype=t.int64, device="cuda")
        crum.hash_pages(b.data_ptr(), b.numel(), out.data_ptr(), stream_handle())
        got = out.cpu().numpy().view(np.uint64)
        exp = oracle.hash_all([h])
        assert np.array_equal(got, exp), f"size {b.numel()}"


def test_hash_pages_special_contents():
    t = torch()
    for fill in [0, 255]:
        b = t.full((5 * P + 100,), fill, dtype=t.uint8, device="cuda")
        out = t.zeros(6, dtype=t.int64, device="cuda")
        crum.hash_pages(b.data_ptr(), b.numel(), out.data_ptr(), stream_handle())
        assert np.array_equal(out.cpu().numpy().view(np.uint64), oracle.hash_all([b.cpu().numpy()]))
    # the all-zero full page has the value pinned from the published sequence
    z = t.zeros(P, dtype=t.uint8, device="cuda")
    out = t.zeros(1, dtype=t.int64, device="cuda")
    crum.hash_pages(z.data_ptr(), P, out.data_ptr(), stream_handle())
    assert int(out.cpu().numpy().view(np.uint64)[0]) == 0xA19D4D208D42E336


@pytest.mark.parametrize("first", [0, 3, 8191, 2**33 + 1])
def test_hash_bytes_matches_oracle(first):
    t = torch()
    for n in [1, 8, 15, 16, 17, 100, 4096, 65536 + 8, 3_000_000 + 3]:
        b = device_buffers([n], seed=n)[0]
        out = t.zeros(1, dtype=t.int64, device="cuda")
        crum.hash_bytes(b.data_ptr(), n, first, out.data_ptr(), stream_handle())
        got = int(out.cpu().numpy().view(np.uint64)[0])
        assert got == oracle.hash_bytes(b.cpu().numpy(), first), n


def _checkpoint_bytes(s, flags=crum.INCR):
    img = s.checkpoint(stream_handle(), flags)
    img.wait(crum.WAIT_PERSISTED)
    return img, img.to_bytes()


def test_small16m_full_incremental_restore():
    """16 MiB fp32, full checkpoint, 10 % of pages rewritten, incremental
    checkpoint, restore of the chain onto garbage."""
    wl = W.workload("small16m")
    bufs = device_buffers(wl.sizes, seed=wl.seed, kind=wl.kind)
    s = make_set(bufs)
    o = oracle.OracleSet(wl.sizes)
    img0, b0 = _checkpoint_bytes(s)
    e0, d0, h0, _ = o.checkpoint(host_copies(bufs))
    assert first_diff(b0, e0) is None
    assert np.array_equal(s.hashes(), h0)
    pages = W.choose_step(wl, 1, wl.n_pages)
    assert pages.size == 26
    W.mutate_pages_(bufs[0], pages, wl.seed + 1)
    img1, b1 = _checkpoint_bytes(s)
    state1 = host_copies(bufs)
    e1, d1, h1, _ = o.checkpoint(state1)
    assert set(np.flatnonzero(d1).tolist()) == set(pages.tolist())
    assert first_diff(b1, e1) is None
    info = img1.info()
    assert info["n_dirty"] == 26 and info["parent_seq"] == 0 and info["full"] == 0
    assert info["checksum"] == int(np.frombuffer(e1[-8:], dtype=np.uint64)[0])
    # restore onto garbage
    W.fill_(bufs[0], 12345, "u32")
    s.restore(img1, stream_handle())
    torch().cuda.synchronize()
    assert np.array_equal(host_copies(bufs)[0], state1[0])
    assert np.array_equal(s.hashes(), h1)
    # after restore, an unchanged state checkpoints empty with the right parent
    img2, b2 = _checkpoint_bytes(s)
    assert parse_header(b2)["n"] == 0 and parse_header(b2)["parent"] == 1
    for i in (img0, img1, img2):
        i.release()
    s.destroy()


def test_ragged_allocations_chain():
    sizes = RAGGED
    bufs = device_buffers(sizes, seed=3)
    s = make_set(bufs)
    o = oracle.OracleSet(sizes)
    chain_dev, states = [], []
    for step in range(4):
        if step:
            touched = mutate(bufs, sizes, 0.3, seed=100 + step)
        img, got = _checkpoint_bytes(s)
        state = host_copies(bufs)
        exp, d, h, _ = o.checkpoint(state)
        if step:
            assert set(np.flatnonzero(d).tolist()) == touched
        assert first_diff(got, exp) is None, f"step {step}"
        chain_dev.append(img)
        states.append(state)
    # restore every prefix of the chain onto garbage
    for k in range(len(chain_dev)):
        for i, b in enumerate(bufs):
            W.fill_(b, 999 + i + k, "u32")
        s.restore(chain_dev[k], stream_handle())
        torch().cuda.synchronize()
        for got, exp in zip(host_copies(bufs), states[k]):
            assert np.array_equal(got, exp), f"prefix {k}"
        assert np.array_equal(s.hashes(), oracle.hash_all(states[k]))
    s.destroy()


def test_empty_and_all_dirty():
    sizes = [5 * P + 3, 2 * P]
    bufs = device_buffers(sizes, seed=5)
    s = make_set(bufs)
    o = oracle.OracleSet(sizes)
    _, b0 = _checkpoint_bytes(s)
    e0, *_ = o.checkpoint(host_copies(bufs))
    assert first_diff(b0, e0) is None
    _, b1 = _checkpoint_bytes(s)
    e1, d1, *_ = o.checkpoint(host_copies(bufs))
    assert d1.sum() == 0 and first_diff(b1, e1) is None
    # explicit FULL: every page, no parent
    _, b2 = _checkpoint_bytes(s, crum.FULL)
    e2, *_ = o.checkpoint(host_copies(bufs), full=True)
    assert first_diff(b2, e2) is None and parse_header(b2)["flags"] == 1
    s.destroy()


@pytest.mark.parametrize("chunk", [0, 3 * 4096 + 8])
def test_chunked_capture_small_staging(chunk):
    """Staging halves of 3 pages: captures run chunk by chunk; with a drain
    copy size that is not a page multiple, every drain is many copies."""
    sizes = [17 * P + 5, 4 * P]
    bufs = device_buffers(sizes, seed=7)
    s = make_set(bufs, staging_bytes=6 * P, chunk_bytes=chunk)
    o = oracle.OracleSet(sizes)
    for step in range(3):
        if step:
            mutate(bufs, sizes, 0.5, seed=70 + step)
        _, got = _checkpoint_bytes(s)
        exp, *_ = o.checkpoint(host_copies(bufs))
        assert first_diff(got, exp) is None, f"step {step}"
    s.destroy()


def test_registration_change_forces_full():
    """Register and unregister between checkpoints: the image after each
    change is full (a new chain base, sequence numbers counting on), the
    one after it incremental again; whole images against the oracle's."""
    sizes = [3 * P, P + 1, 2 * P + 24]
    bufs = device_buffers(sizes, seed=9)
    s = crum.CheckpointSet()
    o = oracle.OracleSet(sizes[:1])
    ids = [s.register(bufs[0].data_ptr(), sizes[0])]
    _, b0 = _checkpoint_bytes(s)
    e0, *_ = o.checkpoint(host_copies(bufs[:1]))
    assert first_diff(b0, e0) is None
    for i in (1, 2):
        ids.append(s.register(bufs[i].data_ptr(), sizes[i]))
        assert o.register(sizes[i]) == ids[-1]
    _, b1 = _checkpoint_bytes(s)
    e1, *_ = o.checkpoint(host_copies(bufs))
    h = parse_header(b1)
    assert h["flags"] == 1 and h["n"] == 3 + 2 + 3 and h["A"] == 3 and h["seq"] == 1
    assert first_diff(b1, e1) is None
    mutate(bufs, sizes, 0.5, seed=91)
    _, b2 = _checkpoint_bytes(s)
    e2, *_ = o.checkpoint(host_copies(bufs))
    assert parse_header(b2)["flags"] == 0 and first_diff(b2, e2) is None
    s.unregister(ids[1])
    o.unregister(ids[1])
    kept = [bufs[0], bufs[2]]
    _, b3 = _checkpoint_bytes(s)
    e3, *_ = o.checkpoint(host_copies(kept))
    assert parse_header(b3)["flags"] == 1 and parse_header(b3)["seq"] == 3
    assert first_diff(b3, e3) is None
    mutate(kept, [sizes[0], sizes[2]], 0.5, seed=92)
    _, b4 = _checkpoint_bytes(s)
    e4, *_ = o.checkpoint(host_copies(kept))
    assert first_diff(b4, e4) is None
    s.destroy()
    s.destroy()


@pytest.mark.parametrize("staging", [0, 4 * P])
def test_verify_mode_reports_injected_collision(staging):
    # staging 4 * P: two slots per half, so the shadow is written chunk by chunk
    sizes = [4 * P + 24]
    bufs = device_buffers(sizes, seed=11)
    s = make_set(bufs, verify=1, staging_bytes=staging)
    o = oracle.OracleSet(sizes)
    _, _ = _checkpoint_bytes(s, crum.VERIFY)
    prev = host_copies(bufs)
    o.checkpoint(prev)
    # change page 2, then make the committed hash equal the new one
    W.mutate_pages_(bufs[0], [2], 77)
    now = host_copies(bufs)
    new_h = int(oracle.hash_all(now)[2])
    s.poke_hash(2, new_h)
    o.h_prev[2] = new_h
    img = s.checkpoint(stream_handle(), crum.VERIFY)
    st = img.wait(crum.WAIT_PERSISTED)
    assert st == crum.ECOLLISION and img.info()["collisions"] == 1
    exp, d, _, coll = o.checkpoint(now, verify_prev=prev)
    assert coll == 1
    assert first_diff(img.to_bytes(), exp) is None
    assert page_table(img.to_bytes()).tolist() == [[0, 2]]
    s.destroy()


@pytest.mark.parametrize("compress", [0, 1])
def test_save_load_corrupt_mismatch(tmp_path, compress):
    sizes = [6 * P + 17]
    bufs = device_buffers(sizes, seed=13, kind="fp32")
    s = make_set(bufs, compress=compress)
    img0, b0 = _checkpoint_bytes(s)
    mutate(bufs, sizes, 0.4, seed=5)
    img1, b1 = _checkpoint_bytes(s)
    state = host_copies(bufs)
    p0, p1 = str(tmp_path / "a.img"), str(tmp_path / "b.img")
    img0.save(p0)
    img1.save(p1)
    s2 = make_set(bufs)
    l0 = s2.load_image(p0)
    l1 = s2.load_image(p1, parent=l0)
    assert l1.info()["n_dirty"] == parse_header(b1)["n"]
    W.fill_(bufs[0], 4242, "u32")
    s2.restore(l1, stream_handle())
    torch().cuda.synchronize()
    assert np.array_equal(host_copies(bufs)[0], state[0])
    # a flipped payload byte, a flipped header byte, a truncated file
    for pos in [len(b1) // 2, 20, len(b1) - 3]:
        bad = bytearray(b1)
        bad[pos] ^= 0x40
        with pytest.raises(crum.CrumError) as e:
            s2.image_from_bytes(bytes(bad), parent=l0)
        assert e.value.status == crum.ECORRUPT
    with pytest.raises(crum.CrumError) as e:
        s2.image_from_bytes(b1[:-16], parent=l0)
    assert e.value.status == crum.ECORRUPT
    # wrong parent
    with pytest.raises(crum.CrumError) as e:
        s2.image_from_bytes(b1, parent=None)
    assert e.value.status == crum.EMISMATCH
    # restore onto a set with a different registration table
    other = device_buffers([6 * P + 16], seed=1)
    s3 = make_set(other)
    with pytest.raises(crum.CrumError) as e:
        s3.restore(img0, stream_handle())
    assert e.value.status == crum.EMISMATCH
    for x in (s, s2, s3):
        x.destroy()


def test_file_sink_writes_each_image(tmp_path):
    sizes = [3 * P + 11]
    bufs = device_buffers(sizes, seed=15)
    s = make_set(bufs, sink=crum.SINK_FILE, sink_dir=str(tmp_path), fsync=1)
    o = oracle.OracleSet(sizes)
    for step in range(3):
        if step:
            mutate(bufs, sizes, 0.5, seed=step)
        img, got = _checkpoint_bytes(s)
        exp, *_ = o.checkpoint(host_copies(bufs))
        files = sorted(os.listdir(tmp_path))
        assert len(files) == step + 1
        name = [f for f in files if f.endswith(f"_{step}.img")][0]
        with open(os.path.join(tmp_path, name), "rb") as f:
            on_disk = f.read()
        assert on_disk == exp == got
    s.destroy()


def test_null_sink_still_counts_pages():
    sizes = [4 * P]
    bufs = device_buffers(sizes, seed=17)
    s = make_set(bufs, sink=crum.SINK_NULL)
    img = s.checkpoint(stream_handle())
    img.wait()
    assert img.info()["n_dirty"] == 4
    with pytest.raises(crum.CrumError):
        img.to_bytes()
    s.destroy()


def test_invalid_registrations():
    t = torch()
    b = t.empty(4 * P, dtype=t.uint8, device="cuda")
    s = crum.CheckpointSet()
    # misaligned, empty, null, and 2^32 pages (past the page table's u32 index)
    for ptr, n in [(b.data_ptr() + 8, P), (b.data_ptr(), 0), (0, P), (b.data_ptr(), (1 << 32) * P)]:
        with pytest.raises(crum.CrumError) as e:
            s.register(ptr, n)
        assert e.value.status == crum.EINVAL
    s.register(b.data_ptr(), 2 * P)
    with pytest.raises(crum.CrumError) as e:
        s.register(b.data_ptr() + P, 2 * P)  # overlaps
    assert e.value.status == crum.EINVAL
    with pytest.raises(crum.CrumError) as e:
        s.checkpoint(stream_handle(), crum.VERIFY)  # set made without verify
    assert e.value.status == crum.EINVAL
    empty = crum.CheckpointSet()
    with pytest.raises(crum.CrumError) as e:
        empty.checkpoint(stream_handle())
    assert e.value.status == crum.EINVAL
    s.destroy()
    empty.destroy()


def test_kernels_are_launched():
    before = crum.kernel_launches()
    bufs = device_buffers([2 * P], seed=19)
    s = make_set(bufs)
    s.checkpoint(stream_handle()).wait()
    assert crum.kernel_launches() - before == 3  # hash, scan, gather
    s.destroy()


@pytest.mark.parametrize("hm", range(crum.NUM_HASH_MAPPINGS))
def test_every_mapping_is_bit_exact(hm):
    """Every autotuner candidate (hash mappings 0-8, gather mappings 0-5)
    gives the oracle's images bit for bit, over ragged allocations."""
    gm = hm % 6
    sizes = RAGGED + [9 * P, 2 * P + 16]
    bufs = device_buffers(sizes, seed=40 + hm)
    s = make_set(bufs, hash_mapping=hm, gather_mapping=gm)
    o = oracle.OracleSet(sizes)
    for step in range(3):
        if step:
            mutate(bufs, sizes, 0.35, seed=400 + 10 * hm + step)
        _, got = _checkpoint_bytes(s)
        exp, *_ = o.checkpoint(host_copies(bufs))
        assert first_diff(got, exp) is None, f"hash {hm} gather {gm} step {step}"
    s.destroy()


def test_autotune_keeps_parity():
    sizes = [40 * P, 3 * P + 8, 17 * P]
    bufs = device_buffers(sizes, seed=51)
    s = make_set(bufs)
    o = oracle.OracleSet(sizes)
    _, b0 = _checkpoint_bytes(s)
    e0, *_ = o.checkpoint(host_copies(bufs))
    assert first_diff(b0, e0) is None
    t = s.autotune()
    assert 0 <= t["hash_mapping"] < crum.NUM_HASH_MAPPINGS and 0 <= t["gather_mapping"] < 6
    assert all(x > 0 for x in t["hash_ms"]) and all(x > 0 for x in t["gather_ms"])
    # autotuning hashed into scratch: the committed hashes are untouched
    assert np.array_equal(s.hashes(), oracle.hash_all(host_copies(bufs)))
    mutate(bufs, sizes, 0.25, seed=52)
    _, b1 = _checkpoint_bytes(s)
    e1, *_ = o.checkpoint(host_copies(bufs))
    assert first_diff(b1, e1) is None
    s.destroy()


@pytest.mark.parametrize("hm", [1, 6])
def test_graph_launch_matches_oracle(hm):
    """Captures launched as one CUDA graph per staging half: same images,
    phase timings recorded, rebuilt after a registration change."""
    sizes = RAGGED + [9 * P]
    bufs = device_buffers(sizes, seed=60 + hm)
    s = make_set(bufs, use_graph=1, hash_mapping=hm)
    o = oracle.OracleSet(sizes)
    for step in range(4):
        if step:
            mutate(bufs, sizes, 0.3, seed=600 + step)
        img, got = _checkpoint_bytes(s)
        exp, *_ = o.checkpoint(host_copies(bufs))
        assert first_diff(got, exp) is None, f"step {step}"
        info = img.info()
        assert info["t_hash_ms"] > 0 and info["t_compact_ms"] > 0
    extra = device_buffers([3 * P + 1], seed=99)
    s.register(extra[0].data_ptr(), extra[0].numel())
    o.register(3 * P + 1)
    for step in range(2):
        if step:
            mutate(bufs + extra, sizes + [3 * P + 1], 0.3, seed=610 + step)
        _, got = _checkpoint_bytes(s)
        exp, *_ = o.checkpoint(host_copies(bufs + extra))
        assert first_diff(got, exp) is None, f"after the change, step {step}"
        assert parse_header(got)["flags"] == (1 if step == 0 else 0)
    s.destroy()


def test_max_chain_bounds_incremental_chains():
    sizes = [6 * P + 9]
    bufs = device_buffers(sizes, seed=71)
    s = make_set(bufs, max_chain=2)
    o = oracle.OracleSet(sizes)
    flags = []
    for step in range(7):
        if step:
            mutate(bufs, sizes, 0.5, seed=710 + step)
        img, got = _checkpoint_bytes(s)
        full = parse_header(got)["flags"] == 1
        exp, *_ = o.checkpoint(host_copies(bufs), full=full)
        assert first_diff(got, exp) is None
        flags.append(int(full))
    assert flags == [1, 0, 0, 1, 0, 0, 1]
    s.destroy()


def test_graph_survives_released_images():
    """Images (and their events) are released between captures; the graph
    path must not refer to them afterwards."""
    sizes = [12 * P + 3]
    bufs = device_buffers(sizes, seed=81)
    s = make_set(bufs, use_graph=1)
    o = oracle.OracleSet(sizes)
    for step in range(6):
        if step:
            mutate(bufs, sizes, 0.4, seed=810 + step)
        img, got = _checkpoint_bytes(s, crum.FULL if step == 3 else crum.INCR)
        exp, *_ = o.checkpoint(host_copies(bufs), full=(step == 3))
        assert first_diff(got, exp) is None, f"step {step}"
        img.release()
    s.destroy()


def test_sink_failure_reports_eio_and_forces_full(tmp_path):
    """A sink that cannot write (host-made failure): the image still drains
    and is correct, PERSISTED reports CRUM_EIO, and the set's next
    checkpoint is full so no chain depends on the unpersisted image."""
    sizes = [5 * P + 1]
    bufs = device_buffers(sizes, seed=91)
    s = make_set(bufs, sink=crum.SINK_FILE, sink_dir=str(tmp_path / "missing" / "dir"))
    o = oracle.OracleSet(sizes)
    img = s.checkpoint(stream_handle())
    assert img.wait(crum.WAIT_PERSISTED, allow=(crum.EIO,)) == crum.EIO
    exp, *_ = o.checkpoint(host_copies(bufs))
    assert first_diff(img.to_bytes(), exp) is None  # drained bytes are intact
    mutate(bufs, sizes, 0.4, seed=92)
    img2 = s.checkpoint(stream_handle())
    img2.wait(crum.WAIT_DRAINED, allow=(crum.OK, crum.EIO))
    assert img2.info()["full"] == 1
    s.destroy()


@pytest.mark.gpu
def test_bounded_wait_runs_out_and_device_stays_usable():
    """A bulk copy that is never issued (a flag nothing sets): the waiting
    consumers give up after the limit, the kernel reports it and returns,
    and the same process then checkpoints bit-exactly."""
    import time
    sizes = [40 * P + 24]
    bufs = device_buffers(sizes, seed=95)
    t0 = time.perf_counter()
    assert crum.selftest_wait_timeout(bufs[0].data_ptr(), bufs[0].numel(), 50_000_000, stream_handle())
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(crum.CrumError):
        crum.selftest_wait_timeout(bufs[0].data_ptr() + 8, bufs[0].numel() - 8, 50_000_000)
    s = make_set(bufs, hash_mapping=6)
    o = oracle.OracleSet(sizes)
    for step in range(2):
        if step:
            mutate(bufs, sizes, 0.3, seed=96)
        img, got = _checkpoint_bytes(s)
        exp, *_ = o.checkpoint(host_copies(bufs))
        assert first_diff(got, exp) is None, f"step {step}"
        img.release()
    s.destroy()


@pytest.mark.gpu
def test_sink_lost_mid_chain_keeps_earlier_images(tmp_path):
    """The writer's directory disappears after two persisted images (the
    host-side stand-in for a writer that died): later images report EIO,
    the two earlier files still load and restore the state they captured."""
    sizes = [9 * P + 5, 3 * P]
    d = tmp_path / "sink"
    d.mkdir()
    bufs = device_buffers(sizes, seed=97)
    s = make_set(bufs, sink=crum.SINK_FILE, sink_dir=str(d))
    states = []
    for step in range(2):
        if step:
            mutate(bufs, sizes, 0.5, seed=98)
        img = s.checkpoint(stream_handle())
        img.wait(crum.WAIT_PERSISTED)
        states.append(host_copies(bufs))
        img.release()
    kept = tmp_path / "kept"
    d.rename(kept)
    mutate(bufs, sizes, 0.5, seed=99)
    img = s.checkpoint(stream_handle())
    assert img.wait(crum.WAIT_PERSISTED, allow=(crum.EIO,)) == crum.EIO
    img.release()
    files = sorted(kept.iterdir(), key=lambda x: int(x.stem.rsplit("_", 1)[1]))
    assert len(files) == 2
    chain = []
    for f, want in zip(files, states):
        chain.append(s.load_image(str(f), chain[-1] if chain else None))
        W.fill_(bufs[0], 4242, "u32")
        W.fill_(bufs[1], 4243, "u32")
        s.restore(chain[-1], stream_handle())
        torch().cuda.synchronize()
        got = host_copies(bufs)
        assert all(np.array_equal(g, w) for g, w in zip(got, want)), f.name
    for c in chain:
        c.release()
    s.destroy()


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [crum.RESTORE_REPLAY, crum.RESTORE_MERGED, crum.RESTORE_AUTO,
                                  crum.RESTORE_DELTA])
def test_chain_restore_forms_agree(mode):
    """Replay (every image in turn) and merged (every page once, from the
    newest image holding it) restore the same bytes and hashes: chain ends
    restored in a non-monotonic order onto garbage, over ragged allocations."""
    sizes = RAGGED
    bufs = device_buffers(sizes, seed=61)
    s = make_set(bufs, restore_mode=mode)
    o = oracle.OracleSet(sizes)
    chain, states, hashes = [], [], []
    for step in range(5):
        if step:
            mutate(bufs, sizes, 0.35, seed=620 + step)
        img = s.checkpoint(stream_handle())
        img.wait()
        chain.append(img)
        states.append(host_copies(bufs))
        _, _, h, _ = o.checkpoint(states[-1])
        hashes.append(h)
    for k in (4, 2, 0, 3):
        for i, b in enumerate(bufs):
            W.fill_(b, 5000 + 17 * k + i, "u32")
        s.restore(chain[k], stream_handle())
        torch().cuda.synchronize()
        got = host_copies(bufs)
        assert all(np.array_equal(g, w) for g, w in zip(got, states[k])), f"chain end {k}"
        assert np.array_equal(s.hashes(), hashes[k]), f"hashes after chain end {k}"
    img = s.checkpoint(stream_handle())
    img.wait()
    info = img.info()
    assert info["n_dirty"] == 0 and info["parent_seq"] == chain[3].info()["seq"]
    img.release()
    for c in chain:
        c.release()
    s.destroy()


@pytest.mark.gpu
def test_merged_restore_of_images_from_bytes():
    """Images rebuilt from their bytes (new pinned buffers) restore through
    the merged form; a chain whose newest image rewrote every page."""
    sizes = [3 * P + 40, 7 * P]
    bufs = device_buffers(sizes, seed=63)
    s = make_set(bufs, restore_mode=crum.RESTORE_MERGED)
    blobs, states = [], []
    for step in range(3):
        if step:
            mutate(bufs, sizes, 1.0 if step == 2 else 0.5, seed=640 + step)
        img, b = _checkpoint_bytes(s)
        blobs.append(b)
        states.append(host_copies(bufs))
        img.release()
    chain = []
    for b in blobs:
        chain.append(s.image_from_bytes(b, chain[-1] if chain else None))
    for i, b in enumerate(bufs):
        W.fill_(b, 6400 + i, "u32")
    s.restore(chain[-1], stream_handle())
    torch().cuda.synchronize()
    assert all(np.array_equal(g, w) for g, w in zip(host_copies(bufs), states[-1]))
    for c in chain:
        c.release()
    s.destroy()


@pytest.mark.gpu
@pytest.mark.parametrize("hm", [0, 1, 2, 3, 4, 5, 9, 10, 11, 12, 13, 14])
def test_verify_mode_collisions_every_mapping(hm):
    """Verify mode over full and tail pages with each register mapping: two
    injected collisions (a full page and a tail page whose committed hash is
    made equal to the new one), one ordinary change, the rest unchanged."""
    sizes = [4 * P, 2 * P + 40]
    bufs = device_buffers(sizes, seed=13)
    s = make_set(bufs, verify=1, hash_mapping=hm)
    o = oracle.OracleSet(sizes)
    _checkpoint_bytes(s, crum.VERIFY)
    prev = host_copies(bufs)
    o.checkpoint(prev)
    W.mutate_pages_(bufs[0], [1, 2], 78)
    W.mutate_pages_(bufs[1], [2], 79)  # the 40-byte tail page
    now = host_copies(bufs)
    h = oracle.hash_all(now)
    for g in (2, 6):  # global pages: allocation 0 page 2, allocation 1 page 2
        s.poke_hash(g, int(h[g]))
        o.h_prev[g] = int(h[g])
    img = s.checkpoint(stream_handle(), crum.VERIFY)
    assert img.wait(crum.WAIT_PERSISTED) == crum.ECOLLISION
    assert img.info()["collisions"] == 2
    exp, d, _, coll = o.checkpoint(now, verify_prev=prev)
    assert coll == 2
    got = img.to_bytes()
    assert first_diff(got, exp) is None
    assert page_table(got).tolist() == [[0, 1], [0, 2], [1, 2]]
    # unchanged since: a verify checkpoint is empty and collision-free
    img2 = s.checkpoint(stream_handle(), crum.VERIFY)
    assert img2.wait(crum.WAIT_PERSISTED) == crum.OK and img2.info()["n_dirty"] == 0
    s.destroy()


@pytest.mark.gpu
def test_delta_restore_moves_only_changed_pages():
    """Rollback: after the chain end, some pages (full and tail) are
    rewritten; a delta restore brings back exactly the chain end's bytes and
    hashes and copies only the rewritten pages across the link, while the
    merged and replay forms copy every page / every image slot."""
    sizes = RAGGED
    bufs = device_buffers(sizes, seed=67)
    n_pages = sum(W.pages_of(n) for n in sizes)
    o = oracle.OracleSet(sizes)
    forms = {m: make_set(bufs, restore_mode=m) for m in
             (crum.RESTORE_DELTA, crum.RESTORE_MERGED, crum.RESTORE_REPLAY)}
    s = forms[crum.RESTORE_DELTA]
    chain = []
    for step in range(3):
        if step:
            mutate(bufs, sizes, 0.3, seed=670 + step)
        img = s.checkpoint(stream_handle())
        img.wait()
        chain.append(img)
    state = host_copies(bufs)
    _, _, h_end, _ = o.checkpoint(state)
    slots = sum(c.info()["n_dirty"] for c in chain)
    for m, r in forms.items():
        touched = mutate(bufs, sizes, 0.1, seed=690 + m)
        r.restore(chain[-1], stream_handle())
        torch().cuda.synchronize()
        assert all(np.array_equal(g, w) for g, w in zip(host_copies(bufs), state)), m
        assert np.array_equal(r.hashes(), h_end), m
        want = {crum.RESTORE_DELTA: len(touched), crum.RESTORE_MERGED: n_pages,
                crum.RESTORE_REPLAY: slots}[m]
        assert r.restore_pages() == want, m
    # nothing changed since: a delta restore copies nothing
    s.restore(chain[-1], stream_handle())
    assert s.restore_pages() == 0
    for c in chain:
        c.release()
    for r in forms.values():
        r.destroy()


@pytest.mark.gpu
@pytest.mark.parametrize("staging", [None, 8 * P])
def test_no_payload_keeps_checksum_and_chain(staging):
    """CRUM_NO_PAYLOAD on a footprint larger than the 64 MiB bounce region,
    through the one-pass and the chunked capture: the image's checksum and
    size equal the oracle's (its payload crossed the link, through several
    bounce copies, and was dropped), and the next incremental, which keeps
    its payload, is byte-exact."""
    sizes = [300 * (1 << 20) + 24]
    bufs = device_buffers(sizes, seed=19)
    s = make_set(bufs, **({} if staging is None else {"staging_bytes": staging}))
    o = oracle.OracleSet(sizes)
    img = s.checkpoint(stream_handle(), crum.FULL | crum.NO_PAYLOAD)
    img.wait()
    exp, *_ = o.checkpoint(host_copies(bufs))
    info = img.info()
    assert info["checksum"] == int(np.frombuffer(exp[-8:], dtype=np.uint64)[0])
    assert info["image_bytes"] == len(exp) and info["n_dirty"] == W.pages_of(sizes[0])
    with pytest.raises(crum.CrumError):
        img.to_bytes()
    mutate(bufs, sizes, 0.05, seed=20)
    img2, got = _checkpoint_bytes(s)
    exp2, *_ = o.checkpoint(host_copies(bufs))
    assert first_diff(got, exp2) is None
    img.release()
    img2.release()
    s.destroy()


@pytest.mark.gpu
def test_max_pending_bounds_unpersisted_images(tmp_path):
    """With max_pending = 1 and a file sink, a checkpoint call returns only
    after the previous image is persisted; every file is the oracle's image."""
    sizes = [6 * P + 8]
    bufs = device_buffers(sizes, seed=23)
    s = make_set(bufs, sink=crum.SINK_FILE, sink_dir=str(tmp_path), max_pending=1)
    o = oracle.OracleSet(sizes)
    imgs, exps = [], []
    for step in range(4):
        if step:
            mutate(bufs, sizes, 0.5, seed=230 + step)
        img = s.checkpoint(stream_handle())
        if imgs:
            assert imgs[-1].info()["stage"] == crum.WAIT_PERSISTED
        imgs.append(img)
        exps.append(o.checkpoint(host_copies(bufs))[0])
    for img, exp in zip(imgs, exps):
        img.wait()
        assert first_diff(img.to_bytes(), exp) is None
        img.release()
    files = sorted(tmp_path.iterdir(), key=lambda x: int(x.stem.rsplit("_", 1)[1]))
    assert [f.read_bytes() for f in files] == exps
    s.destroy()


def test_twenty_thousand_small_allocations():
    # 20,000 allocations of 1 byte to 3 pages carved from one buffer (16-byte
    # aligned, with gaps): the allocation table, the flattened page list and
    # the gather's search over allocations at five times the large
    # workload's count; full, incremental, restore onto scribbled memory
    t = torch()
    rng = np.random.default_rng(2020)
    sizes = [int(x) for x in rng.integers(1, 3 * P, size=20000)]
    gaps = rng.integers(0, 4, size=len(sizes)) * 16
    offs, at = [], 0
    for n, g in zip(sizes, gaps):
        offs.append(at)
        at += (n + 15) // 16 * 16 + int(g)
    big = t.empty(at, dtype=t.uint8, device="cuda")
    W.fill_(big, 2021, "u32")
    bufs = [big[o:o + n] for o, n in zip(offs, sizes)]

    def state():
        h = big.cpu().numpy()
        return [h[o:o + n].copy() for o, n in zip(offs, sizes)]

    s = make_set(bufs)
    o = oracle.OracleSet(sizes)
    img0, got = _checkpoint_bytes(s)
    s0 = state()
    exp, *_ = o.checkpoint(s0)
    assert first_diff(got, exp) is None
    # rewrite the first page of every seventh allocation
    touched = list(range(0, len(sizes), 7))
    for i in touched:
        W.mutate_pages_(bufs[i], np.array([0]), 2022 + i)
    t.cuda.synchronize()
    img1, got = _checkpoint_bytes(s)
    s1 = state()
    exp, d, _, _ = o.checkpoint(s1)
    assert first_diff(got, exp) is None
    assert parse_header(got)["n"] == int(np.count_nonzero(d)) == len(touched)
    W.fill_(big, 2023, "u32")
    s.restore(img1, stream_handle())
    t.cuda.synchronize()
    assert all(np.array_equal(g, e) for g, e in zip(state(), s1))
    img0.release()
    img1.release()
    s.destroy()
