"""Position-keyed tables S_tau (Section 3.1) on the GPU: a disk sector matches a master sector
only at the same position in an 8-sector cluster, clusters counted from the scan's base_offset.
The expected result is the oracle's: the byte-equality definition filtered by
((i - base_offset) mod 8) == (s mod 8)."""
import ctypes

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


def position_workload(seed, n_sectors=20000, n_files=40):
    """The generator's workload shifted by 3 sectors (planted clusters off the 8-sector grid),
    with master sectors copied to other positions inside and across files and scattered over
    the image at arbitrary positions."""
    plan = synth.config_plan(f"small:{n_sectors}:{n_files}:{seed}")
    files = plan.masters_host()
    img = plan.image_host()
    rng = np.random.default_rng(seed)
    for _ in range(40):
        f, g = (int(x) for x in rng.integers(0, len(files), 2))
        nf, ng = files[f].size // SECTOR, files[g].size // SECTOR
        if nf and ng:
            s, t = int(rng.integers(0, nf)), int(rng.integers(0, ng))
            files[g][t * SECTOR:(t + 1) * SECTOR] = files[f][s * SECTOR:(s + 1) * SECTOR]
    secs = img.reshape(-1, SECTOR)
    for _ in range(400):
        f = int(rng.integers(0, len(files)))
        nf = files[f].size // SECTOR
        if nf:
            s = int(rng.integers(0, nf))
            secs[int(rng.integers(0, secs.shape[0]))] = files[f][s * SECTOR:(s + 1) * SECTOR]
    head = rng.integers(0, 256, 3 * SECTOR, dtype=np.uint8)
    return np.concatenate([head, img]), files


@pytest.mark.parametrize("sig", [0, 1, 2, 3])
@pytest.mark.parametrize("base", [0, 3, 11, (1 << 40) + 5])
def test_position_scan_equals_oracle(cv, sig, base):
    img, files = position_workload(90 + sig)
    want = oracle.match_position(img, files, base)
    full = oracle.match_hash(img, files)
    assert 0 < want.size < full.size  # the filter is selective on this input
    with cv.master_build(files, signature=sig, position_mode=cv.CV_POSITION_CLUSTER) as m:
        info = m.info()
        assert info["position_mode"] == cv.CV_POSITION_CLUSTER and info["signature"] == sig
        dev = torch.from_numpy(img).cuda()
        with cv.scan(m, [dev], base_offset=base) as r:
            assert np.array_equal(r.matches(0), want)
        # host image streamed in chunks that start off the cluster grid
        with cv.scan(m, [img], chunk_bytes=1001 * SECTOR, base_offset=base) as r:
            assert np.array_equal(r.matches(0), want)


def test_position_many_images_count_from_their_own_start(cv):
    img, files = position_workload(97)
    cuts = [(0, 7001), (7001, 7002), (7002, 12345), (12345, img.size // SECTOR)]
    dev = torch.from_numpy(img).cuda()
    with cv.master_build(files, position_mode=cv.CV_POSITION_CLUSTER) as m:
        for base in (0, 6):
            images = []
            for k, (a, b) in enumerate(cuts):
                images.append(dev[a * SECTOR:b * SECTOR] if k % 2 == 0 else np.ascontiguousarray(img[a * SECTOR:b * SECTOR]))
            with cv.scan(m, images, base_offset=base) as r:
                for k, (a, b) in enumerate(cuts):
                    want = oracle.match_position(img[a * SECTOR:b * SECTOR], files, base)
                    assert np.array_equal(r.matches(k), want), (base, k)


@pytest.mark.parametrize("max_load,bloom", [(0.9, 0), (0.9, 16), (0.25, 8)])
def test_position_table_options(cv, max_load, bloom):
    img, files = position_workload(98)
    want = oracle.match_position(img, files, 5)
    with cv.master_build(files, max_load=max_load, bloom_bits_per_key=bloom,
                         position_mode=cv.CV_POSITION_CLUSTER) as m:
        with cv.scan(m, [torch.from_numpy(img).cuda()], base_offset=5) as r:
            assert np.array_equal(r.matches(0), want)


def test_position_info_and_any_table(cv):
    """The keyed table holds one key per distinct (digest, tau); the same masters without
    positions still give the unfiltered result."""
    img, files = position_workload(99)
    with cv.master_build(files, position_mode=cv.CV_POSITION_CLUSTER) as mp, cv.master_build(files) as ma:
        ip, ia = mp.info(), ma.info()
        assert ia["position_mode"] == cv.CV_POSITION_ANY
        assert ip["n_kept"] == ia["n_kept"]
        kept = set()
        for f in files:
            for s in range(f.size // SECTOR):
                sec = f[s * SECTOR:(s + 1) * SECTOR]
                if not oracle.sector_trivial(sec):
                    kept.add((sec.tobytes(), s % 8))
        assert ip["n_unique"] == len(kept)
        assert ia["n_unique"] == len({k for k, _ in kept})
        dev = torch.from_numpy(img).cuda()
        with cv.scan(ma, [dev], base_offset=3) as r:  # ignored without positions
            assert np.array_equal(r.matches(0), oracle.match_hash(img, files))


def test_position_batch_server_noalloc(cv):
    img, files = position_workload(100)
    dev = torch.from_numpy(img).cuda()
    cuts = [(0, 5003), (5003, 5004), (5004, img.size // SECTOR)]
    wants = [oracle.match_position(img[a * SECTOR:b * SECTOR], files, 0) for a, b in cuts]
    with cv.master_build(files, position_mode=cv.CV_POSITION_CLUSTER) as m:
        with cv.batch_create(m, [(dev.data_ptr() + a * SECTOR, (b - a) * SECTOR) for a, b in cuts]) as b:
            b.run()
            b.wait()
            for k in range(len(cuts)):
                assert np.array_equal(cv.device_matches_to_numpy(b.matches(k)), wants[k])
        with cv.server_create(m, work_unit_bytes=1001 * SECTOR, hbm_budget_bytes=8 << 20) as srv:
            ts = [srv.submit(np.ascontiguousarray(img[a * SECTOR:b * SECTOR])) for a, b in cuts]
            for k, t in enumerate(ts):
                r = srv.poll(t, timeout_ms=60000)
                assert np.array_equal(r.matches(0), wants[k])
                r.close()


def test_position_mode_rejected_and_old_struct_sizes(cv):
    lib = cv.load()
    h = ctypes.c_void_p()
    o = cv.cv_master_opts(ctypes.sizeof(cv.cv_master_opts), 0.0, 0, 0, None, 2, 0)
    assert lib.cv_master_build(None, 0, ctypes.byref(o), ctypes.byref(h)) == cv.CV_EINVAL
    img, files = position_workload(101, n_sectors=4096, n_files=10)
    arr, keep = cv._bufs(files)
    o = cv.cv_master_opts(24, 0.0, cv.CV_BLOOM_AUTO, 0, None, 1, 0)  # without position_mode: ANY
    assert lib.cv_master_build(arr, len(files), ctypes.byref(o), ctypes.byref(h)) == cv.CV_OK
    m = cv.Master(h.value)
    assert m.info()["position_mode"] == cv.CV_POSITION_ANY
    m.close()
