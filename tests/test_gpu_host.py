"""Pinned host memory from cv_host_alloc: aligned to the huge page size and backed by huge
pages where the kernel allows them, zeroed, known to the CUDA driver as pinned, released
exactly once; and every scan path reading an image from it (cv_scan,
chunked cv_scan, the serving loop) gives the oracle's matches bit for bit."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAGE = 4096


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def driver_knows_pinned(p: int) -> bool:
    """cuMemHostGetFlags succeeds only for page-locked memory the driver knows (allocated or
    registered); it needs the current context, which torch has made current."""
    drv = ctypes.CDLL("libcuda.so.1")
    flags = ctypes.c_uint()
    return drv.cuMemHostGetFlags(ctypes.byref(flags), ctypes.c_void_p(p)) == 0


def huge_page_bytes():
    try:
        return int(open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size").read())
    except OSError:
        return 2 << 20


def thp_mode():
    try:
        s = open("/sys/kernel/mm/transparent_hugepage/enabled").read()
        return s[s.index("[") + 1:s.index("]")]
    except (OSError, ValueError):
        return "never"


def anon_huge_kib(p: int) -> int:
    """AnonHugePages of the mapping that holds address p, from /proc/self/smaps."""
    lines = open("/proc/self/smaps").read().split("\n")
    for i, line in enumerate(lines):
        head = line.split()
        if head and "-" in head[0]:
            try:
                lo, hi = (int(x, 16) for x in head[0].split("-"))
            except ValueError:
                continue
            if lo <= p < hi:
                for x in lines[i + 1:i + 40]:
                    if x.startswith("AnonHugePages:"):
                        return int(x.split()[1])
    return 0


def test_alloc_is_aligned_zeroed_and_pinned(cv):
    torch.cuda.init()
    plain = (ctypes.c_uint8 * PAGE)()
    assert not driver_knows_pinned(ctypes.addressof(plain))
    huge = huge_page_bytes()
    n = 2 * huge + 123
    with cv.host_alloc(n) as hb:
        assert hb.ptr % huge == 0
        assert driver_knows_pinned(hb.ptr) and driver_knows_pinned(hb.ptr + n - 1)
        if thp_mode() != "never":
            # backed by huge pages (the kernel may fall short on a fragmented host: half at least)
            assert anon_huge_kib(hb.ptr) * 1024 >= 3 * huge // 2, anon_huge_kib(hb.ptr)
        a = hb.array()
        assert a.size == n and not a.any()
        t = torch.from_numpy(a)
        a[:] = 7
        d = t.cuda(non_blocking=True)
        torch.cuda.synchronize()
        assert int(d.sum()) == 7 * a.size


def test_alloc_and_free_errors(cv):
    lib = cv.load()
    p = ctypes.c_void_p()
    assert lib.cv_host_alloc(0, ctypes.byref(p)) == cv.CV_EINVAL and not p.value
    assert lib.cv_host_alloc(PAGE, None) == cv.CV_EINVAL
    assert lib.cv_host_free(None) == cv.CV_OK
    assert lib.cv_host_alloc(PAGE, ctypes.byref(p)) == cv.CV_OK and p.value
    assert lib.cv_host_free(p.value + PAGE // 2) == cv.CV_EINVAL  # not a block start
    assert lib.cv_host_free(p.value) == cv.CV_OK
    assert lib.cv_host_free(p.value) == cv.CV_EINVAL  # already released
    buf = (ctypes.c_uint8 * PAGE)()
    assert lib.cv_host_free(ctypes.addressof(buf)) == cv.CV_EINVAL  # not from cv_host_alloc


def test_scans_from_host_alloc_match_the_oracle(cv):
    plan = synth.config_plan("small:40000:40:83")
    img = plan.image_host()
    files = plan.masters_host()
    want = oracle.match_hash(img, files)
    assert want.size
    with cv.host_alloc(img.nbytes) as hb:
        hb.array()[:] = img
        with cv.master_build(files) as m:
            with cv.scan(m, [(hb.ptr, img.nbytes)]) as r:
                assert np.array_equal(r.matches(0), want)
            # chunked: the image crosses several 1 MiB copies
            with cv.scan(m, [(hb.ptr, img.nbytes)] * 2, chunk_bytes=1 << 20) as r:
                assert np.array_equal(r.matches(0), want) and np.array_equal(r.matches(1), want)
            with cv.server_create(m, work_unit_bytes=1 << 20, copy_streams=2, max_copy_bytes=2 << 20) as srv:
                t = [srv.submit((hb.ptr, img.nbytes), tag=k) for k in range(3)]
                for k in range(3):
                    r = srv.poll(t[k], timeout_ms=-1)
                    assert np.array_equal(r.matches(0), want)
                    r.close()
