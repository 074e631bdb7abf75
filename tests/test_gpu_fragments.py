"""Fragment scans on the GPU (Section 5: every 64-byte window at a 4-byte offset against the
64-byte fragments of the master files), bit-exact against the oracle: every supported
signature and table layout, Bloom filter on and off, host and device images, ragged image
lengths, windows across tile boundaries, shared fragments and djb2 collisions."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth
from test_oracle_fragments import tricky_frag_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FRAG = 64
SIGS = [0, 1, 2]  # MD5, MD5 without padding, djb2-64
TILE_BYTES = 256 * 33 * 4  # bytes between the starts of two fragment tiles


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def frag_master(cv, files, sig=0, **kw):
    return cv.master_build(files, signature=sig, unit=cv.CV_UNIT_FRAGMENT, **kw)


def dev(img):
    # copy into a 16-byte aligned device buffer
    t = torch.empty(max(img.size, 1), dtype=torch.uint8, device="cuda")
    if img.size:
        t[: img.size].copy_(torch.from_numpy(img))
    return (t.data_ptr(), img.size), t


@pytest.mark.parametrize("sig", SIGS)
@pytest.mark.parametrize("layout", [0, 1])
def test_tricky_cases(cv, sig, layout):
    for seed in range(6):
        image, files = tricky_frag_case(seed)
        want = oracle.frag_match(image, files)
        for bloom in (0, 16):
            with frag_master(cv, files, sig, layout=layout, bloom_bits_per_key=bloom) as m:
                d, keep = dev(image)
                with cv.scan(m, [d, image]) as r:
                    assert np.array_equal(r.matches(0), want), (seed, bloom)
                    assert np.array_equal(r.matches(1), want), (seed, bloom)


def generated(seed, n_bytes, n_logos, header_frac=0.3):
    fp = synth.make_frag_plan(seed, n_bytes, n_logos, header_frac=header_frac)
    return fp, fp.image_host(), fp.logos()


@pytest.mark.parametrize("sig", SIGS)
def test_generated_workload_and_ragged_images(cv, sig):
    fp, img, logos = generated(60 + sig, (6 << 20) + 13, 300)
    want = oracle.frag_match(img, logos)
    assert want.size > 1000
    exp = fp.expected_planted()
    with frag_master(cv, logos, sig) as m:
        info = m.info()
        assert info["unit"] == cv.CV_UNIT_FRAGMENT
        assert info["n_sectors"] == sum(x.size // FRAG for x in logos)
        d, keep = dev(img)
        with cv.scan(m, [d]) as r:
            got = r.matches(0)
            assert np.array_equal(got, want)
            assert r.stats()["sectors"] == (img.size - FRAG) // 4 + 1
        gs = set(map(tuple, got.tolist()))
        assert set(map(tuple, exp.tolist())) <= gs
        # ragged lengths: tails inside a 16-byte chunk, a tile boundary, shorter than a window
        cuts = [0, 63, 64, 65, 67, TILE_BYTES - 1, TILE_BYTES + 64, TILE_BYTES + 77, 3 * TILE_BYTES + 5, img.size]
        pieces = [np.ascontiguousarray(img[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
        bufs, keeps = [], []
        for k, pc in enumerate(pieces):
            if k % 2:
                bufs.append(pc)
            else:
                b, t = dev(pc)
                bufs.append(b)
                keeps.append(t)
        with cv.scan(m, bufs) as r:
            for k, pc in enumerate(pieces):
                assert np.array_equal(r.matches(k), oracle.frag_match(pc, logos)), k


def test_windows_across_tile_boundaries(cv):
    """Copies whose windows straddle the end of a tile (the next tile's first windows and the
    64 staged bytes past a tile's last window start)."""
    rng = np.random.default_rng(5)
    logo = rng.integers(0, 256, 1000, dtype=np.uint8)
    img = rng.integers(0, 256, 5 * TILE_BYTES, dtype=np.uint8)
    for o in (TILE_BYTES - 60, 2 * TILE_BYTES - 4, 3 * TILE_BYTES - 64, 4 * TILE_BYTES - 992):
        img[o:o + logo.size] = logo
    want = oracle.frag_match(img, [logo])
    assert want.size == 4 * (1000 // FRAG)
    for sig in SIGS:
        with frag_master(cv, [logo], sig) as m:
            d, keep = dev(img)
            with cv.scan(m, [d]) as r:
                assert np.array_equal(r.matches(0), want), sig


def test_djb2_collisions_are_confirmed(cv):
    rng = np.random.default_rng(8)
    logos = [rng.integers(40, 200, 64 * 20, dtype=np.uint8) for _ in range(5)]
    img = rng.integers(0, 256, 1 << 20, dtype=np.uint8)
    pos = 0
    for f, lg in enumerate(logos):
        for j in range(0, 20, 3):
            frag = lg[j * FRAG:(j + 1) * FRAG].copy()
            col = frag.copy()
            col[7] += 1
            col[8] -= 33  # same djb2-64, other bytes
            assert oracle.djb2_64(col) == oracle.djb2_64(frag)
            pos += 4096
            img[pos:pos + FRAG] = col
            img[pos + 1000:pos + 1000 + FRAG] = frag
    want = oracle.frag_match(img, logos)
    # candidates the confirmation must drop: windows whose djb2 equals a kept fragment's while
    # their bytes differ
    wsig = oracle.window_signatures(img, 2)[:, :8].copy().view("<u8").ravel()
    frags = {}
    for lg in logos:
        for j in range(lg.size // FRAG):
            fr = lg[j * FRAG:(j + 1) * FRAG]
            if not oracle.fragment_trivial(fr):
                frags.setdefault(oracle.djb2_64(fr), []).append(fr)
    rejected = 0
    for k in np.nonzero(np.isin(wsig, np.array(list(frags), dtype=np.uint64)))[0]:
        w = img[4 * k:4 * k + FRAG]
        rejected += sum(int(not np.array_equal(w, fr)) for fr in frags[int(wsig[k])])
    assert rejected >= 35
    with frag_master(cv, logos, 2) as m:
        d, keep = dev(img)
        with cv.scan(m, [d]) as r:
            assert np.array_equal(r.matches(0), want)
            assert r.stats()["confirm_rejected"] == rejected
    assert want.size == sum(len(range(0, 20, 3)) for _ in logos)


def test_fragment_shared_by_many_files(cv):
    rng = np.random.default_rng(9)
    header = rng.integers(0, 256, 128, dtype=np.uint8)
    logos = [np.concatenate([header, rng.integers(0, 256, 256, dtype=np.uint8)]) for _ in range(400)]
    img = rng.integers(0, 256, 1 << 19, dtype=np.uint8)
    for o in (100, 50000, 300000):
        o -= o % 4
        img[o:o + logos[7].size] = logos[7]
    want = oracle.frag_match(img, logos)
    assert want.size == 3 * (2 * 400 + 4)
    for sig in SIGS:
        for layout in (0, 1):
            with frag_master(cv, logos, sig, layout=layout) as m:
                d, keep = dev(img)
                with cv.scan(m, [d], keep_on_device=True) as r:
                    assert np.array_equal(cv.device_matches_to_numpy(r.matches(0)), want)


def test_fragment_64mib_against_oracle(cv):
    fp, img, logos = generated(77, 64 << 20, 2000, header_frac=0.1)
    want = oracle.frag_match(img, logos)
    with frag_master(cv, logos, 2) as m:
        t = torch.empty(img.size, dtype=torch.uint8, device="cuda")
        fp.image_device(torch, t)
        assert np.array_equal(t.cpu().numpy(), img)  # the device generator writes the same bytes
        with cv.scan(m, [t]) as r:
            assert np.array_equal(r.matches(0), want)


def test_fragment_rejections(cv):
    rng = np.random.default_rng(10)
    logos = [rng.integers(0, 256, 640, dtype=np.uint8)]
    for kw in ({"signature": 3}, {"position_mode": cv.CV_POSITION_CLUSTER}):
        with pytest.raises(cv.CVError) as e:
            cv.master_build(logos, unit=cv.CV_UNIT_FRAGMENT, **kw)
        assert e.value.code == cv.CV_EINVAL
    img = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    with frag_master(cv, logos) as m:
        with pytest.raises(cv.CVError):
            cv.batch_create(m, [img])
        with pytest.raises(cv.CVError):
            cv.server_create(m)
        out = torch.empty(1 << 12, dtype=torch.uint8, device="cuda")
        rc, _ = cv.scan_noalloc(m, img, out, 256, check=False)
        assert rc == cv.CV_EINVAL
    lib = cv.load()
    o = cv.cv_master_opts(ctypes.sizeof(cv.cv_master_opts), 0.0, 0, 0, None, 0, 0, 2, 0)
    h = ctypes.c_void_p()
    assert lib.cv_master_build(None, 0, ctypes.byref(o), ctypes.byref(h)) == cv.CV_EINVAL


@pytest.mark.parametrize("sig", SIGS)
def test_empty_fragment_tables(cv, sig):
    """Fragment tables without a single kept fragment (no files, an empty file, a file shorter
    than a fragment, only all-equal fragments) find nothing, for every layout and filter."""
    rng = np.random.default_rng(12)
    img = rng.integers(0, 256, 50_000, dtype=np.uint8)
    d, keep = dev(img)
    for files in ([], [np.zeros(0, np.uint8)], [rng.integers(0, 256, 63, dtype=np.uint8)],
                  [np.zeros(640, np.uint8), np.full(128, 7, np.uint8)]):
        for layout in (0, 1):
            for bloom in (0, 16):
                with frag_master(cv, files, sig, layout=layout, bloom_bits_per_key=bloom) as m:
                    with cv.scan(m, [d, img]) as r:
                        assert r.matches(0).size == 0 and r.matches(1).size == 0
