"""Saved tables: every kind of table saved and loaded back scans exactly like the table it came
from (and like the oracle); damaged or foreign files are refused with an error code, including a
slot whose posting range points past the postings (checked on the device at load time)."""
import ctypes
import struct

import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def header_bytes(cv):
    """The table file's header: tag, version, size, the info struct, 10 words, 6 byte counts."""
    return 8 + 4 + 4 + ctypes.sizeof(cv.cv_master_info) + 10 * 4 + 6 * 8


KINDS = [
    dict(),
    dict(layout=1, position_mode=1),
    dict(signature=2),
    dict(signature=3, layout=1, bloom_bits_per_key=0),
    dict(signature=1, max_load=0.9),
]


@pytest.mark.parametrize("kw", KINDS)
def test_save_load_round_trip(cv, kw, tmp_path):
    plan = synth.config_plan("small:16000:30:81")
    img = plan.image_host()
    files = plan.masters_host()
    dev = torch.from_numpy(img).cuda()
    want = oracle.match_position(img, files, 0) if kw.get("position_mode") else oracle.match_hash(img, files)
    path = tmp_path / "t.cvt"
    with cv.master_build(files, **kw) as m:
        cv.master_save(m, path)
        info = m.info()
    with cv.master_load(path) as m2:
        assert m2.info() == info
        with cv.scan(m2, [dev]) as r:
            assert np.array_equal(r.matches(0), want)


def test_save_load_fragments_and_empty(cv, tmp_path):
    fp = synth.make_frag_plan(82, 1 << 20, 30, header_frac=0.3)
    img = fp.image_host()
    logos = fp.logos()
    path = tmp_path / "f.cvt"
    with cv.master_build(logos, signature=2, unit=cv.CV_UNIT_FRAGMENT) as m:
        cv.master_save(m, path)
    with cv.master_load(path) as m2, cv.scan(m2, [torch.from_numpy(img).cuda()]) as r:
        assert np.array_equal(r.matches(0), oracle.frag_match(img, logos))
    empty = tmp_path / "e.cvt"
    with cv.master_build([np.zeros(1024, np.uint8)]) as m:
        cv.master_save(m, empty)
    with cv.master_load(empty) as m2, cv.scan(m2, [torch.from_numpy(img).cuda()]) as r:
        assert r.matches(0).size == 0


def test_damaged_files_refused(cv, tmp_path):
    plan = synth.config_plan("small:4000:10:83")
    files = plan.masters_host()
    path = tmp_path / "t.cvt"
    with cv.master_build(files) as m:
        cv.master_save(m, path)
        n_slots = m.info()["n_slots"]
    data = bytearray(path.read_bytes())
    HEADER = header_bytes(cv)
    assert struct.unpack_from("<I", data, 12)[0] == HEADER

    def refused(blob, code):
        bad = tmp_path / "bad.cvt"
        bad.write_bytes(bytes(blob))
        with pytest.raises(cv.CVError) as e:
            cv.master_load(bad)
        assert e.value.code == code

    refused(data[:HEADER - 5], cv.CV_EIO)            # header cut short
    refused(data[:-7], cv.CV_EIO)                     # arrays cut short
    refused(data + b"x", cv.CV_ECORRUPT)              # trailing bytes
    bad = bytearray(data)
    bad[0] ^= 1
    refused(bad, cv.CV_ECORRUPT)                      # not a table file
    bad = bytearray(data)
    struct.pack_into("<I", bad, 8, 99)
    refused(bad, cv.CV_ECORRUPT)                      # unknown version
    # an occupied slot whose posting range runs past the postings
    slots = np.frombuffer(bytes(data[HEADER:HEADER + 32 * n_slots]), np.uint32).reshape(-1, 8)
    k = int(np.nonzero(slots[:, 5])[0][0])
    bad = bytearray(data)
    struct.pack_into("<I", bad, HEADER + 32 * k + 20, 0x7FFFFFFF)
    refused(bad, cv.CV_ECORRUPT)
    with pytest.raises(cv.CVError) as e:
        cv.master_load(tmp_path / "missing.cvt")
    assert e.value.code == cv.CV_EIO
