"""cv_scan_noalloc: the scan entry point for callers that must not allocate memory while they
work (fixed-buffer ingest loops, processes whose device memory is reserved up front). It uses a
scratch array built into the library instead of a memory pool; its results must equal the
regular cv_scan entry point's, call after call, even though every call reuses the same array.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

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
    with cv.master_build(files) as m:
        want_a = _regular(cv, m, a)
        want_b = _regular(cv, m, b)
        assert want_a.size > want_b.size > 0
        got_a = _noalloc(cv, m, a, want_a.size + 10)
        got_b = _noalloc(cv, m, b, want_b.size + 10)
        assert np.array_equal(got_a, want_a)
        assert np.array_equal(got_b, want_b)


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
