"""The sorted table layout (binary search, the alternative to linear probing that Section 4
suggests for high occupancy) gives the same results as the hash layout and the oracle: every
signature, with and without positions and Bloom filter, empty and one-key tables, and keys
whose first word is equal (so the search lands on a run of equal first words)."""
import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth
from test_oracle_signatures import crc_high_twin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def layout_workload(seed):
    plan = synth.config_plan(f"small:16384:40:{seed}")
    files = plan.masters_host()
    img = plan.image_host()
    rng = np.random.default_rng(seed)
    secs = img.reshape(-1, SECTOR)
    # first-word twins under CRC64: x and y are master sectors, z only on the disk
    f = files[0]
    x = f[:SECTOR].copy()
    y, z = crc_high_twin(x, 1), crc_high_twin(x, 2)
    f[SECTOR:2 * SECTOR] = y
    for s in (x, y, z):
        for _ in range(3):
            secs[int(rng.integers(0, secs.shape[0]))] = s
    return img, files


@pytest.mark.parametrize("sig", [0, 1, 2, 3])
@pytest.mark.parametrize("position", [0, 1])
def test_sorted_equals_oracle(cv, sig, position):
    img, files = layout_workload(120 + sig)
    want = oracle.match_position(img, files, 3) if position else oracle.match_hash(img, files)
    dev = torch.from_numpy(img).cuda()
    for bloom in (0, 16):
        with cv.master_build(files, signature=sig, position_mode=position, layout=cv.CV_LAYOUT_SORTED,
                             bloom_bits_per_key=bloom) as m:
            info = m.info()
            assert info["layout"] == cv.CV_LAYOUT_SORTED
            assert info["n_slots"] == info["n_unique"]
            assert info["max_probe"] == int(np.ceil(np.log2(info["n_unique"])))
            with cv.scan(m, [dev], base_offset=3) as r:
                assert np.array_equal(r.matches(0), want), bloom
            with cv.scan(m, [img], chunk_bytes=777 * SECTOR, base_offset=3) as r:
                assert np.array_equal(r.matches(0), want), bloom


def test_sorted_equal_first_words_with_crc(cv):
    """x and y share the first key word and are both in the table; z shares it and is not."""
    img, files = layout_workload(130)
    want = oracle.match_hash(img, files)
    x, y = files[0][:SECTOR], files[0][SECTOR:2 * SECTOR]
    assert oracle.crc64(x) & 0xFFFFFFFF == oracle.crc64(y) & 0xFFFFFFFF
    with cv.master_build(files, signature=3, layout=cv.CV_LAYOUT_SORTED, bloom_bits_per_key=0) as m:
        with cv.scan(m, [torch.from_numpy(img).cuda()]) as r:
            got = r.matches(0)
    assert np.array_equal(got, want)
    hit_files = {(int(t["file_id"]), int(t["file_sector"])) for t in got}
    assert (0, 0) in hit_files and (0, 1) in hit_files


def test_sorted_degenerate_tables(cv):
    img = synth.random_sectors(5, 64)
    dev = torch.from_numpy(img).cuda()
    with cv.master_build([np.zeros(4 * SECTOR, np.uint8)], layout=cv.CV_LAYOUT_SORTED) as m:  # nothing kept
        assert m.info()["n_unique"] == 0
        with cv.scan(m, [dev]) as r:
            assert r.matches(0).size == 0
    one = img[7 * SECTOR:8 * SECTOR].copy()
    with cv.master_build([one], layout=cv.CV_LAYOUT_SORTED) as m:  # one key: no search step
        assert m.info()["n_unique"] == 1 and m.info()["max_probe"] == 0
        with cv.scan(m, [dev]) as r:
            assert np.array_equal(r.matches(0), oracle.match_hash(img, [one]))
    with cv.master_build([], layout=cv.CV_LAYOUT_SORTED) as m:
        with cv.scan(m, [dev]) as r:
            assert r.matches(0).size == 0


def test_sorted_batch_server_noalloc(cv):
    img, files = layout_workload(131)
    dev = torch.from_numpy(img).cuda()
    cuts = [(0, 3001), (3001, 16384)]
    wants = [oracle.match_hash(img[a * SECTOR:b * SECTOR], files) for a, b in cuts]
    with cv.master_build(files, layout=cv.CV_LAYOUT_SORTED) as m:
        with cv.batch_create(m, [(dev.data_ptr() + a * SECTOR, (b - a) * SECTOR) for a, b in cuts],
                             autotune=1) as b:
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
        out = torch.empty(16 * (wants[1].size + 8), dtype=torch.uint8, device="cuda")
        a, bnd = cuts[1]
        rc, n = cv.scan_noalloc(m, (dev.data_ptr() + a * SECTOR, (bnd - a) * SECTOR), out, wants[1].size + 8)
        assert rc == cv.CV_OK and n == wants[1].size
        assert np.array_equal(np.frombuffer(out[: n * 16].cpu().numpy().tobytes(), cv.MATCH_DTYPE), wants[1])


@pytest.mark.parametrize("max_load,bloom", [(0.9, 0), (0.9, 16), (0.5, 0), (0.25, 16)])
def test_auto_layout_follows_occupancy(cv, max_load, bloom):
    img, files = layout_workload(140)
    want = oracle.match_hash(img, files)
    with cv.master_build(files, max_load=max_load, bloom_bits_per_key=bloom) as mh:
        occ = mh.info()["n_unique"] / mh.info()["n_slots"]
    with cv.master_build(files, max_load=max_load, bloom_bits_per_key=bloom, layout=cv.CV_LAYOUT_AUTO) as m:
        expect = cv.CV_LAYOUT_SORTED if occ > (0.8 if bloom else 0.5) else cv.CV_LAYOUT_HASH
        assert m.info()["layout"] == expect, occ
        with cv.scan(m, [torch.from_numpy(img).cuda()]) as r:
            assert np.array_equal(r.matches(0), want)
