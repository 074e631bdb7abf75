"""cv_probe_profile: the table reads of a scan's lookups, counted on the GPU, against counts
derived here from hashlib's MD5 and the table rules (Eq. 3 linear probing; bisection for the
sorted layout).

The hash-layout pin rests on two facts of linear probing that hold whatever order the GPU
inserted the keys in: the set of occupied slots, and the total displacement of the stored keys,
depend only on the keys' home slots. So the reads of a missing key (its walk up to the first
empty slot, cut at the probe bound) and the summed reads of every stored key looked up once
are both fixed by the homes alone."""
import ctypes
import hashlib
import struct

import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth
from probe_model import linear_probing_model, miss_reads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def d0_of(sector: bytes) -> int:
    """Word 0 of the MD5 digest (bytes 0-3, little-endian): the home-slot key of Eq. 3."""
    return struct.unpack("<I", hashlib.md5(sector).digest()[:4])[0]


def sectors_of(a: np.ndarray):
    return [a[i * SECTOR:(i + 1) * SECTOR].tobytes() for i in range(a.size // SECTOR)]


@pytest.mark.parametrize("max_load,seed", [(0.9, 1), (0.5, 2), (0.9, 3)])
def test_hash_layout_reads_exact(cv, max_load, seed):
    rng = np.random.default_rng(seed)
    masters = rng.integers(0, 256, 700 * SECTOR, dtype=np.uint8)
    misses = rng.integers(0, 256, 3000 * SECTOR, dtype=np.uint8)
    image = np.concatenate([misses[:1500 * SECTOR], masters, misses[1500 * SECTOR:]])
    with cv.master_build([masters], bloom_bits_per_key=0, max_load=max_load) as m:
        info = m.info()
        n_slots = info["n_slots"]
        homes = [d0_of(s) & (n_slots - 1) for s in sectors_of(masters)]
        occ, total, _ = linear_probing_model(homes, n_slots)
        # the longest displacement, hence the probe bound, depends on the insertion order: the
        # table's own bound cuts the walks
        bound = info["max_probe"]
        assert 1 <= bound <= n_slots
        want_reads = total + sum(miss_reads(occ, d0_of(s) & (n_slots - 1), bound) for s in sectors_of(misses))
        got = cv.probe_profile(m, torch.from_numpy(image).cuda())
    assert got == {"layout": 0, "sectors": 3700, "bloom_passed": 3700, "slot_reads": want_reads, "key_reads": 0,
                   "found": 700}


def sorted_lookup_model(keys, h0, present):
    """Key words and records read by a lookup of h0 in the sorted key words (distinct here);
    present: the sector's full key is stored (else a record with an equal h0 fails to compare
    and the next key word is read too)."""
    n = len(keys)
    reads, base, m = 0, 0, n
    while m > 1:
        half = m >> 1
        reads += 1
        base = base + half if keys[base + half] < h0 else base
        m -= half
    reads += 1
    j = base + (1 if keys[base] < h0 else 0)
    records = 0
    if j < n:
        reads += 1
        if keys[j] == h0:
            records = 1
            if not present and j + 1 < n:
                reads += 1
    return reads, records


def test_sorted_layout_reads_exact(cv):
    rng = np.random.default_rng(4)
    masters = rng.integers(0, 256, 900 * SECTOR, dtype=np.uint8)
    misses = rng.integers(0, 256, 2000 * SECTOR, dtype=np.uint8)
    image = np.concatenate([masters, misses])
    keys = sorted(d0_of(s) for s in sectors_of(masters))
    assert len(set(keys)) == len(keys)
    want_keys = want_slots = 0
    stored = set(sectors_of(masters))
    for s in sectors_of(image):
        k, r = sorted_lookup_model(keys, d0_of(s), s in stored)
        want_keys += k
        want_slots += r
    with cv.master_build([masters], bloom_bits_per_key=0, layout=1) as m:
        assert m.info()["layout"] == 1
        got = cv.probe_profile(m, torch.from_numpy(image).cuda())
    assert got == {"layout": 1, "sectors": 2900, "bloom_passed": 2900, "slot_reads": want_slots,
                   "key_reads": want_keys, "found": 900}


def test_bloom_only_removes_lookups(cv):
    """With a Bloom filter: the same keys are found, fewer sectors reach the table, and no
    more slots are read than without one."""
    plan = synth.config_plan("small:30000:40:61")
    files = plan.masters_host()
    img = plan.image_host()
    dev = torch.from_numpy(img).cuda()
    hit_sectors = np.unique(oracle.match_hash(img, files)["disk_sector"]).size
    with cv.master_build(files) as mb, cv.master_build(files, bloom_bits_per_key=0) as mn:
        a = cv.probe_profile(mb, dev)
        b = cv.probe_profile(mn, dev)
    assert a["found"] == b["found"] == hit_sectors > 0
    assert b["bloom_passed"] == b["sectors"] == 30000
    assert a["found"] <= a["bloom_passed"] < b["bloom_passed"]
    assert a["bloom_passed"] <= a["slot_reads"] <= b["slot_reads"]


@pytest.mark.parametrize("sig", [0, 2, 3])
@pytest.mark.parametrize("base", [0, 5])
def test_position_tables_and_signatures_find_the_oracles_sectors(cv, sig, base):
    plan = synth.config_plan("small:20000:30:62")
    files = plan.masters_host()
    img = plan.image_host()
    want = np.unique(oracle.match_position(img, files, base)["disk_sector"]).size
    with cv.master_build(files, signature=sig, position_mode=1) as m:
        got = cv.probe_profile(m, torch.from_numpy(img).cuda(), base_offset=base)
    # 64-bit signatures count key matches before byte confirmation: at least the true ones
    assert got["found"] == want if sig == 0 else got["found"] >= want
    assert got["sectors"] == 20000 and got["slot_reads"] >= got["bloom_passed"] >= got["found"]


def test_errors_and_empty(cv):
    files = [synth.random_sectors(5, 64)]
    lib = cv.load()
    img = torch.from_numpy(np.ascontiguousarray(files[0])).cuda()
    with cv.master_build(files) as m:
        assert cv.probe_profile(m, (img.data_ptr(), 0))["sectors"] == 0
        st = cv.cv_probe_stats()
        st.struct_size = ctypes.sizeof(st) - 8
        assert lib.cv_probe_profile(m.handle, img.data_ptr(), SECTOR, 0, ctypes.byref(st), None) == cv.CV_EINVAL
        st.struct_size = ctypes.sizeof(st)
        assert lib.cv_probe_profile(m.handle, img.data_ptr() + 4, SECTOR, 0, ctypes.byref(st), None) == cv.CV_EINVAL
        host = np.ascontiguousarray(files[0])
        assert lib.cv_probe_profile(m.handle, host.ctypes.data, SECTOR, 0, ctypes.byref(st), None) == cv.CV_EINVAL
        assert lib.cv_probe_profile(None, img.data_ptr(), SECTOR, 0, ctypes.byref(st), None) == cv.CV_EINVAL
    fp = synth.make_frag_plan(83, 1 << 16, 4)
    with cv.master_build(fp.logos(), unit=1, signature=2) as mf:
        assert lib.cv_probe_profile(mf.handle, img.data_ptr(), SECTOR, 0, ctypes.byref(st), None) == cv.CV_EINVAL
