"""cv_scan_noalloc: the scan entry point for callers that must not allocate memory while they
work (fixed-buffer ingest loops, processes whose device memory is reserved up front). It uses a
scratch array built into the library instead of a memory pool; its results must equal the
regular cv_scan entry point's, call after call, even though every call reuses the same array.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def _regular(cv, master, img_t):
    with cv.scan(master, [img_t]) as r:
        return r.matches(0)


def _noalloc(cv, master, img_t, capacity):
    out = torch.empty(max(capacity, 1) * 16, dtype=torch.uint8, device="cuda")
    rc, n = cv.scan_noalloc(master, img_t, out, capacity)
    assert rc == cv.CV_OK
    got = np.frombuffer(out[: n * 16].cpu().numpy().tobytes(), cv.MATCH_DTYPE)
    return got


def test_noalloc_equals_regular_scan_two_calls_in_a_row(cv):
    plan_a = synth.config_plan("small:300001:200:41")  # ragged size, many matches
    plan_b = synth.make_plan(42, 70000, plan_a.file_nsect, 0.05, master_seed=plan_a.master_seed)
    files = plan_a.masters_host()
    a = torch.from_numpy(plan_a.image_host()).cuda()
    b = torch.from_numpy(plan_b.image_host()).cuda()
    # the definition's result, from the oracle
    ora_a = oracle.match_hash(plan_a.image_host(), files)
    ora_b = oracle.match_hash(plan_b.image_host(), files)
    with cv.master_build(files) as m:
        want_a = _regular(cv, m, a)
        want_b = _regular(cv, m, b)
        assert want_a.size > want_b.size > 0
        assert np.array_equal(want_a, ora_a) and np.array_equal(want_b, ora_b)
        got_a = _noalloc(cv, m, a, want_a.size + 10)
        got_b = _noalloc(cv, m, b, want_b.size + 10)
        assert np.array_equal(got_a, ora_a)
        assert np.array_equal(got_b, ora_b)


def test_noalloc_allocates_no_device_memory(cv):
    """After one call (which does the per-device set-up), further calls of different sizes leave
    the device's free memory and torch's reserved memory exactly where they were."""
    plan = synth.config_plan("small:120000:80:44")
    files = plan.masters_host()
    img = torch.from_numpy(plan.image_host()).cuda()
    want = oracle.match_hash(plan.image_host(), files)
    out = torch.empty((want.size + 16) * 16, dtype=torch.uint8, device="cuda")
    with cv.master_build(files) as m:
        rc, n = cv.scan_noalloc(m, img, out, want.size + 16)
        assert rc == cv.CV_OK and n == want.size
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        for sectors in (120000, 1, 4097, 77777, 120000):
            rc, n = cv.scan_noalloc(m, (img.data_ptr(), sectors * SECTOR), out, want.size + 16)
            assert rc == cv.CV_OK
            assert n == int(np.searchsorted(want["disk_sector"], sectors))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_reserved() == reserved0
        got = np.frombuffer(out[: n * 16].cpu().numpy().tobytes(), cv.MATCH_DTYPE)
        assert np.array_equal(got, want)


def test_noalloc_refuses_a_capturing_stream(cv):
    plan = synth.config_plan("small:4096:10:45")
    files = plan.masters_host()
    img = torch.from_numpy(plan.image_host()).cuda()
    want = oracle.match_hash(plan.image_host(), files)
    cap = want.size + 8
    out = torch.empty(16 * cap, dtype=torch.uint8, device="cuda")
    with cv.master_build(files) as m:
        rc, n = cv.scan_noalloc(m, img, out, cap)  # set-up outside any capture
        assert rc == cv.CV_OK and n == want.size
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            try:
                rc, _ = cv.scan_noalloc(m, img, out, cap, stream=s, check=False)
            finally:
                g.capture_end()
        assert rc == cv.CV_EINVAL
        out.zero_()
        rc, n = cv.scan_noalloc(m, img, out, cap)
        assert rc == cv.CV_OK
        assert np.array_equal(np.frombuffer(out[: n * 16].cpu().numpy().tobytes(), cv.MATCH_DTYPE), want)


def test_noalloc_limits(cv):
    plan = synth.config_plan("small:20000:30:43")
    files = plan.masters_host()
    img = torch.from_numpy(plan.image_host()).cuda()
    with cv.master_build(files) as m:
        want = _regular(cv, m, img)
        assert want.size > 2
        # too little room: only the first entries are written, the full count is reported
        out = torch.zeros(16 * 2, dtype=torch.uint8, device="cuda")
        rc, n = cv.scan_noalloc(m, img, out, 2)
        assert rc == cv.CV_ERANGE and n == want.size
        assert np.array_equal(np.frombuffer(out.cpu().numpy().tobytes(), cv.MATCH_DTYPE), want[:2])
        # an image above the fixed scratch limit is refused before any work
        rc, n = cv.scan_noalloc(m, (img.data_ptr(), (cv.CV_NOALLOC_MAX_SECTORS + 1) * SECTOR), out, 2, check=False)
        assert rc == cv.CV_EINVAL
        # and the next regular-sized call is still right
        assert np.array_equal(_noalloc(cv, m, img, want.size), want)
