"""crum_dirty_pages_static: the allocation-free way to ask which pages of
one allocation changed, for callers that cannot call cudaMalloc when they
need the answer (an out-of-memory handler taking a last checkpoint, an
allocator hook or CUDA-call interposer that must not re-enter the
allocator).  Its scratch is a fixed device array inside the library.

Checked through the C ABI against the regular path (crum_checkpoint's page
table and the set's committed hashes) and against the oracle (its page
hashes and dirty rule) on calls made back to back, so the second call runs
over what the first left in the shared scratch.  The file
name makes pytest collect it last."""
import numpy as np
import pytest

import oracle
import paper_1808_00117_b300 as crum
from paper_1808_00117_b300 import workloads as W

from helpers import device_buffers, make_set, page_table, stream_handle, torch

pytestmark = pytest.mark.gpu
P = 65536


@pytest.fixture(autouse=True)
def _cuda():
    if not torch().cuda.is_available():
        pytest.skip("needs a CUDA device")
    crum.load()


def _static_call(buf, hashes, full):
    t = torch()
    n = W.pages_of(buf.numel())
    pages = t.full((n,), -1, dtype=t.int32, device="cuda")
    count = t.full((1,), -1, dtype=t.int64, device="cuda")
    st = crum.load().crum_dirty_pages_static(buf.data_ptr(), buf.numel(), hashes.data_ptr(),
                                             int(full), pages.data_ptr(), count.data_ptr(),
                                             stream_handle())
    assert st == crum.OK, crum.load().crum_last_error()
    t.cuda.synchronize()
    c = int(count.item())
    return pages[:c].cpu().numpy().view(np.uint32).astype(np.int64), c


def test_static_matches_checkpoint_on_consecutive_calls():
    t = torch()
    size = 300 * P + 4104
    buf = device_buffers([size], seed=21)[0]
    n = W.pages_of(size)
    s = make_set([buf])
    hashes = t.zeros(n, dtype=t.int64, device="cuda")

    # call 1: full listing, hashes from zero
    img0 = s.checkpoint(stream_handle())
    img0.wait()
    h_prev = np.zeros(n, dtype=np.uint64)
    got_pages, c = _static_call(buf, hashes, full=True)
    exp_pages = page_table(img0.to_bytes())[:, 1].astype(np.int64)
    assert c == n and np.array_equal(got_pages, exp_pages)
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), s.hashes())
    # and against the oracle directly: its page hashes and its dirty rule
    host = buf.cpu().numpy()
    h_exp = oracle.hash_all([host])
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), h_exp)
    d_exp, _ = oracle.dirty(h_exp, h_prev, None, True)
    assert np.array_equal(got_pages, np.flatnonzero(d_exp))
    h_prev = h_exp

    # call 2, straight after: incremental over the scratch call 1 left behind
    W.mutate_pages_(buf, W.choose_uniform(5, n, 97), 6)
    img1 = s.checkpoint(stream_handle())
    img1.wait()
    got_pages, c = _static_call(buf, hashes, full=False)
    exp_pages = page_table(img1.to_bytes())[:, 1].astype(np.int64)
    assert c == img1.info()["n_dirty"] == 97
    assert np.array_equal(got_pages, exp_pages)
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), s.hashes())
    host = buf.cpu().numpy()
    h_exp = oracle.hash_all([host])
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), h_exp)
    d_exp, _ = oracle.dirty(h_exp, h_prev, None, False)
    assert np.array_equal(got_pages, np.flatnonzero(d_exp))

    # call 3: nothing changed, nothing listed
    _, c = _static_call(buf, hashes, full=False)
    assert c == 0
    img0.release()
    img1.release()
    s.destroy()


@pytest.mark.parametrize("n_full, tail, k", [(1100, 100, 300), (32768, 4104, 2000)],
                         ids=["1101_pages", "32769_pages"])
def test_static_matches_checkpoint_many_warps(n_full, tail, k):
    """Sizes whose bitmap spreads over several warps of the listing kernel
    (1,101 pages: 35 bitmap words) and over more words than it has threads
    (32,769 pages, just over 2 GiB: 1,025 words, two per thread), with the
    changed pages scattered over the whole allocation and the tail page
    among them; two calls back to back, checked against the regular path."""
    t = torch()
    size = n_full * P + tail
    buf = device_buffers([size], seed=23)[0]
    n = W.pages_of(size)
    s = make_set([buf], staging_bytes=2 * (k + 8) * P, sink=crum.SINK_NULL)
    hashes = t.zeros(n, dtype=t.int64, device="cuda")
    s.checkpoint(stream_handle(), crum.FULL | crum.NO_PAYLOAD).wait()
    _, c = _static_call(buf, hashes, full=True)
    assert c == n
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), s.hashes())
    for rnd in range(2):
        chosen = np.union1d(W.choose_uniform(40 + rnd, n, k), [n - 1])
        W.mutate_pages_(buf, chosen, 50 + rnd)
        img = s.checkpoint(stream_handle())
        img.wait()
        got_pages, c = _static_call(buf, hashes, full=False)
        info = img.info()
        assert c == info["n_dirty"] == chosen.size
        assert np.array_equal(got_pages, chosen)
        assert np.array_equal(hashes.cpu().numpy().view(np.uint64), s.hashes())
        img.release()
    s.destroy()


def test_static_rejects_more_pages_than_its_scratch():
    t = torch()
    buf = t.empty(P, dtype=t.uint8, device="cuda")
    # checked before any device work; the last size is one whose page count
    # wraps past 2^64 when rounded up
    for too_many in ((4194304 + 1) * P, 4194304 * P + 1, 2**64 - 1, 2**64 - P + 1):
        st = crum.load().crum_dirty_pages_static(buf.data_ptr(), too_many, buf.data_ptr(), 0,
                                                 buf.data_ptr(), buf.data_ptr(), stream_handle())
        assert st == crum.EINVAL, too_many
        assert b"CRUM_STATIC_MAX_PAGES" in crum.load().crum_last_error()
