"""crum_dirty_pages_static: the allocation-free way to ask which pages of
one allocation changed, for callers that cannot call cudaMalloc when they
need the answer (an out-of-memory handler taking a last checkpoint, an
allocator hook or CUDA-call interposer that must not re-enter the
allocator).  Its scratch is a fixed device array inside the library.

Checked through the C ABI against the regular path (crum_checkpoint's page
table and the set's committed hashes) on calls made back to back, so the
second call runs over what the first left in the shared scratch.  The file
name makes pytest collect it last."""
import numpy as np
import pytest

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
    got_pages, c = _static_call(buf, hashes, full=True)
    exp_pages = page_table(img0.to_bytes())[:, 1].astype(np.int64)
    assert c == n and np.array_equal(got_pages, exp_pages)
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), s.hashes())

    # call 2, straight after: incremental over the scratch call 1 left behind
    W.mutate_pages_(buf, W.choose_uniform(5, n, 97), 6)
    img1 = s.checkpoint(stream_handle())
    img1.wait()
    got_pages, c = _static_call(buf, hashes, full=False)
    exp_pages = page_table(img1.to_bytes())[:, 1].astype(np.int64)
    assert c == img1.info()["n_dirty"] == 97
    assert np.array_equal(got_pages, exp_pages)
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), s.hashes())

    # call 3: nothing changed, nothing listed
    _, c = _static_call(buf, hashes, full=False)
    assert c == 0
    img0.release()
    img1.release()
    s.destroy()


def test_static_rejects_more_pages_than_its_scratch():
    t = torch()
    buf = t.empty(P, dtype=t.uint8, device="cuda")
    too_many = (4194304 + 1) * P  # checked before any device work
    st = crum.load().crum_dirty_pages_static(buf.data_ptr(), too_many, buf.data_ptr(), 0,
                                             buf.data_ptr(), buf.data_ptr(), stream_handle())
    assert st == crum.EINVAL
    assert b"CRUM_STATIC_MAX_PAGES" in crum.load().crum_last_error()
