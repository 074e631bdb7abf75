"""The paper's other sector signatures on the GPU: MD5 without the padding block, djb2 with a
64-bit accumulator (Eq. 1) and CRC64. 64-bit signatures collide, so the library confirms every
candidate byte for byte; with real collisions planted in the inputs the result must still equal
the byte-equality definition (and the oracle's signature route) exactly."""
import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth
from test_oracle_signatures import crc_collision, djb2_collision

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512
SIGS = [1, 2, 3]


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def workload_with_collisions(seed):
    plan = synth.config_plan(f"small:20000:40:{seed}")
    files = plan.masters_host()
    img = plan.image_host()
    secs = img.reshape(-1, SECTOR)
    rng = np.random.default_rng(seed)
    for k in range(40):  # collide with random master sectors under both 64-bit signatures
        f = int(rng.integers(0, len(files)))
        s = int(rng.integers(0, files[f].size // SECTOR))
        m = files[f][s * SECTOR:(s + 1) * SECTOR].copy()
        m[:] = np.clip(m, 40, 200)  # keep room for the +1/-33 djb2 construction
        files[f][s * SECTOR:(s + 1) * SECTOR] = m
        secs[int(rng.integers(0, secs.shape[0]))] = djb2_collision(m, 17)
        secs[int(rng.integers(0, secs.shape[0]))] = crc_collision(m, 1001)
        secs[int(rng.integers(0, secs.shape[0]))] = m  # and a true match
    return img, files


def expected_rejected(img, files, sig):
    """Candidates the byte confirmation must drop: (disk sector, kept master sector) pairs whose
    signatures (the oracle's) are equal while their bytes differ."""
    if sig not in (2, 3):
        return 0
    by_sig = {}
    for f in files:
        secs = f[: f.size // SECTOR * SECTOR].reshape(-1, SECTOR)
        sigs = oracle.signatures(secs, sig)[:, :8].copy().view("<u8").ravel()
        for s, h in zip(secs, sigs):
            if not oracle.sector_trivial(s):
                by_sig.setdefault(int(h), []).append(s)
    disk = img[: img.size // SECTOR * SECTOR].reshape(-1, SECTOR)
    dsig = oracle.signatures(disk, sig)[:, :8].copy().view("<u8").ravel()
    n = 0
    for d, h in zip(disk, dsig):
        for s in by_sig.get(int(h), ()):
            n += int(not np.array_equal(d, s))
    return n


@pytest.mark.parametrize("sig", SIGS)
def test_scan_signature_equals_definition(cv, sig):
    img, files = workload_with_collisions(70 + sig)
    want = oracle.match_brute(img, files)
    assert np.array_equal(oracle.match_sig(img, files, sig), want)
    rejected = expected_rejected(img, files, sig)
    if sig in (2, 3):
        assert rejected >= 35  # the planted collisions (a few overwritten by later plants) reach it
    with cv.master_build(files, signature=sig) as m:
        assert m.info()["signature"] == sig
        with cv.scan(m, [torch.from_numpy(img).cuda()]) as r:
            assert np.array_equal(r.matches(0), want)
            assert r.stats()["confirm_rejected"] == rejected
        with cv.scan(m, [img], chunk_bytes=1 << 20) as r:  # host image
            assert np.array_equal(r.matches(0), want)
            assert r.stats()["confirm_rejected"] == rejected


@pytest.mark.parametrize("sig", SIGS)
def test_batch_server_noalloc_with_signature(cv, sig):
    img, files = workload_with_collisions(80 + sig)
    whole = torch.from_numpy(img).cuda()
    cuts = [(0, 5000), (5000, 5001), (5001, 20000)]
    wants = [oracle.match_brute(img[a * SECTOR:b * SECTOR], files) for a, b in cuts]
    with cv.master_build(files, signature=sig) as m:
        images = [(whole.data_ptr() + a * SECTOR, (b - a) * SECTOR) for a, b in cuts]
        with cv.batch_create(m, images) as b:
            b.run()
            b.wait()
            for k in range(len(cuts)):
                assert np.array_equal(cv.device_matches_to_numpy(b.matches(k)), wants[k])
        with cv.server_create(m, work_unit_bytes=1 << 20, hbm_budget_bytes=4 << 20) as srv:
            ts = [srv.submit(np.ascontiguousarray(img[a * SECTOR:b * SECTOR])) for a, b in cuts]
            for k, t in enumerate(ts):
                r = srv.poll(t, timeout_ms=60000)
                assert np.array_equal(r.matches(0), wants[k])
                r.close()
        out = torch.empty(16 * (wants[2].size + 8), dtype=torch.uint8, device="cuda")
        a, bnd = cuts[2]
        rc, n = cv.scan_noalloc(m, (whole.data_ptr() + a * SECTOR, (bnd - a) * SECTOR), out, wants[2].size + 8)
        assert rc == cv.CV_OK and n == wants[2].size
        assert np.array_equal(np.frombuffer(out[: n * 16].cpu().numpy().tobytes(), cv.MATCH_DTYPE), wants[2])
