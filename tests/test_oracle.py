"""Pins for the CPU oracle, against things other than itself (no GPU needed).

* MD5: Python's hashlib (OpenSSL) and the md5sum tool, two independent implementations, on
  every length class that exercises padding (0..300 bytes, block edges, long inputs) and on
  every sector class the workloads hold (random, zero, fill, text).
* The matching result: a pure-Python statement of the definition (byte-equal sectors, trivial
  master sectors excluded, whole sectors only) on tiny inputs built to hold duplicates, fills,
  partial tails and empty files; and the generator's plant log at the tiny workload's full size.
"""
import hashlib
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

SECTOR = 512


def py_match(image: bytes, files) -> list:
    """The definition, in plain Python: every (i, f, s) with equal bytes, trivial masters out."""
    by_bytes = {}
    for f, data in enumerate(files):
        for s in range(len(data) // SECTOR):
            sec = bytes(data[s * SECTOR:(s + 1) * SECTOR])
            if len(set(sec)) == 1:
                continue
            by_bytes.setdefault(sec, []).append((f, s))
    out = []
    for i in range(len(image) // SECTOR):
        for f, s in by_bytes.get(bytes(image[i * SECTOR:(i + 1) * SECTOR]), []):
            out.append((i, f, s))
    return sorted(out)


def as_list(arr) -> list:
    return [(int(a), int(b), int(c)) for a, b, c in zip(arr["disk_sector"], arr["file_id"], arr["file_sector"])]


# --------------------------------------------------------------------------------- MD5


def test_md5_matches_hashlib_all_padding_lengths():
    rng = np.random.default_rng(123)
    for length in list(range(0, 301)) + [447, 448, 511, 512, 513, 1023, 1024, 4095, 4096, 4097, 65536 + 7]:
        data = rng.integers(0, 256, length, dtype=np.uint8).tobytes()
        assert oracle.md5(data) == hashlib.md5(data).digest(), length


def test_md5_matches_hashlib_structured_inputs():
    cases = [b"", b"\x00" * 512, b"\xff" * 512, bytes(range(256)) * 2, b"\x80" + b"\x00" * 511,
             b"a" * 1000, b"\x00" * 55, b"\x00" * 56, b"\xff" * 64]
    for d in cases:
        assert oracle.md5(d) == hashlib.md5(d).digest()


def test_md5_matches_md5sum_tool():
    rng = np.random.default_rng(7)
    with tempfile.TemporaryDirectory() as td:
        for k, length in enumerate([0, 3, 512, 4096, 100000]):
            data = rng.integers(0, 256, length, dtype=np.uint8).tobytes()
            path = os.path.join(td, f"f{k}")
            with open(path, "wb") as fh:
                fh.write(data)
            out = subprocess.run(["md5sum", path], check=True, capture_output=True, text=True).stdout
            assert out.split()[0] == oracle.md5(data).hex()


def test_md5_sectors_every_sector_class():
    plan = synth.config_plan("small:2048:10:5")
    img = plan.image_host()
    dg = oracle.md5_sectors(img)
    assert dg.shape == (2048, 16)
    for i in range(0, 2048, 7):
        assert dg[i].tobytes() == hashlib.md5(img[i * SECTOR:(i + 1) * SECTOR].tobytes()).digest()
    # the image holds all three background classes and planted sectors
    secs = img.reshape(-1, SECTOR)
    zero = (secs == 0).all(axis=1)
    text = ((secs >= 97) & (secs <= 122) | (secs == 32)).all(axis=1)
    assert zero.sum() > 100 and text.sum() > 100


# ---------------------------------------------------------------------- exclusion rule


def test_trivial_rule():
    assert oracle.sector_trivial(np.zeros(SECTOR, np.uint8))
    assert oracle.sector_trivial(np.full(SECTOR, 0x41, np.uint8))
    assert oracle.sector_trivial(np.full(SECTOR, 0xFF, np.uint8))
    for pos in (0, 1, 255, 510, 511):
        s = np.zeros(SECTOR, np.uint8)
        s[pos] = 1
        assert not oracle.sector_trivial(s), pos
    text = np.frombuffer((b"ab " * 200)[:SECTOR], np.uint8)
    assert not oracle.sector_trivial(text)


# -------------------------------------------------------------------- match definition


def tricky_case(seed: int):
    """A tiny image and master set holding every degenerate case of the definition."""
    rng = np.random.default_rng(seed)
    rnd = lambda n: rng.integers(0, 256, n * SECTOR, dtype=np.uint8)
    shared = rnd(3)  # sectors shared by several files
    files = []
    a = rnd(6)
    a[SECTOR:2 * SECTOR] = 0                       # all-zero master sector: excluded
    a[3 * SECTOR:4 * SECTOR] = 0x5A                # one-byte fill: excluded
    a[4 * SECTOR:5 * SECTOR] = shared[:SECTOR]
    files.append(a)
    b = np.concatenate([shared, shared[:SECTOR], rnd(1)[:100]])  # duplicate inside a file + partial tail
    files.append(b)
    files.append(np.zeros(0, np.uint8))            # empty file
    files.append(rnd(1)[:300])                     # smaller than a sector: no whole sector
    c = rnd(2)
    c[10] ^= 1
    files.append(c)
    near = np.zeros(SECTOR, np.uint8)
    near[511] = 7                                  # all zero but one byte: kept
    files.append(near)
    text = np.frombuffer((b"lorem ipsum dolor " * 40)[:SECTOR], np.uint8).copy()
    files.append(text)
    pieces = []
    for k in range(40):
        r = rng.integers(0, 9)
        if r == 0:
            pieces.append(np.zeros(SECTOR, np.uint8))
        elif r == 1:
            pieces.append(np.full(SECTOR, 0x5A, np.uint8))
        elif r == 2:
            pieces.append(shared[SECTOR * rng.integers(0, 3):][:SECTOR])
        elif r == 3:
            f = files[rng.integers(0, 2)]
            s = rng.integers(0, f.size // SECTOR)
            pieces.append(f[s * SECTOR:(s + 1) * SECTOR])
        elif r == 4:
            pieces.append(near)
        elif r == 5:
            pieces.append(text)
        elif r == 6:
            x = c[:SECTOR].copy()
            x[10] ^= 1                             # one bit off a master sector: no match
            pieces.append(x)
        else:
            pieces.append(rnd(1))
    pieces.append(shared[:200])                    # trailing partial sector: ignored
    image = np.concatenate(pieces)
    return image, files


@pytest.mark.parametrize("seed", range(12))
def test_brute_and_hash_equal_definition(seed):
    image, files = tricky_case(seed)
    want = py_match(image.tobytes(), [f.tobytes() for f in files])
    assert len(want) > 0
    assert as_list(oracle.match_brute(image, files)) == want
    assert as_list(oracle.match_hash(image, files)) == want


def test_empty_inputs():
    files = [np.zeros(0, np.uint8)]
    assert oracle.match_hash(np.zeros(0, np.uint8), files).size == 0
    assert oracle.match_brute(np.zeros(100, np.uint8), files).size == 0
    img = synth.random_sectors(1, 4)
    assert oracle.match_hash(img, []).size == 0
    assert oracle.match_hash(img, [img]).size == 4


def test_hash_on_generated_small_workloads():
    for seed in range(3):
        plan = synth.config_plan(f"small:4096:24:{seed + 10}")
        img = plan.image_host()
        files = plan.masters_host()
        got = oracle.match_hash(img, files)
        assert np.array_equal(got, oracle.match_brute(img, files))
        assert np.array_equal(got, plan.expected_intact())
        assert got.size > 50


def test_db_lookup_any_window_equals_whole_scan():
    plan = synth.config_plan("small:8192:30:21")
    img = plan.image_host()
    files = plan.masters_host()
    whole = oracle.match_hash(img, files)
    db = oracle.OracleDB(files)
    assert len(db) == plan.n_master_sectors
    for first, n in [(0, 8192), (5, 1000), (4096, 4096), (8191, 1)]:
        got = db.lookup(img[first * SECTOR:(first + n) * SECTOR], first)
        sel = whole[(whole["disk_sector"] >= first) & (whole["disk_sector"] < first + n)]
        assert np.array_equal(got, sel)


def test_tiny_workload_plant_log():
    """The 64 MiB workload at full size: every intact planted sector is found, nothing else."""
    plan = synth.config_plan("tiny")
    img = plan.image_host()
    files = plan.masters_host()
    got = oracle.match_hash(img, files)
    exp = plan.expected_intact()
    assert exp.size > 10000
    assert np.array_equal(got, exp)
    # every reported pair is byte-equal
    secs = img.reshape(-1, SECTOR)
    for t in got[:: max(1, got.size // 500)]:
        f = files[t["file_id"]]
        s = int(t["file_sector"])
        assert np.array_equal(secs[t["disk_sector"]], f[s * SECTOR:(s + 1) * SECTOR])


@pytest.mark.parametrize("base", [0, 3, 8, 13])
def test_position_keyed_matching(base):
    """S_tau restricts the result to equal cluster positions: the definition's triples filtered
    by ((i - base) mod 8) == (s mod 8); planted whole clusters all survive at base 0 and none at
    a base that is not a multiple of 8."""
    plan = synth.config_plan("small:8192:20:31")
    img = plan.image_host()
    files = plan.masters_host()
    want = [t for t in py_match(img.tobytes(), [f.tobytes() for f in files]) if (t[0] - base) % 8 == t[2] % 8]
    got = as_list(oracle.match_position(img, files, base))
    assert got == want
    full = oracle.match_hash(img, files)
    if base % 8 == 0:
        assert got == as_list(full)
    else:
        assert got == []
    image, files2 = tricky_case(2)
    want2 = [t for t in py_match(image.tobytes(), [f.tobytes() for f in files2]) if (t[0] - base) % 8 == t[2] % 8]
    assert as_list(oracle.match_position(image, files2, base)) == want2
