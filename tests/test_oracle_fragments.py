"""Pins for the oracle's fragment matching (Section 5: every 64-byte window at a 4-byte offset of
the image against the 64-byte fragments of the master files), on the CPU.

* Both oracle routes against a pure-Python statement of the definition on tiny inputs built to
  hold every degenerate case: windows that end exactly at the image end, images shorter than
  a window or not a multiple of 4 bytes long, partial tail fragments, all-equal fragments,
  fragments shared by several files and repeated inside one, planted copies at every residue
  of the offset modulo 64.
* The generator's plant log on generated workloads.
"""
import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

FRAG, STRIDE = 64, 4


def py_frag_match(image: bytes, files) -> list:
    """The definition in plain Python."""
    by_bytes = {}
    for f, data in enumerate(files):
        for j in range(len(data) // FRAG):
            fr = bytes(data[j * FRAG:(j + 1) * FRAG])
            if len(set(fr)) == 1:
                continue
            by_bytes.setdefault(fr, []).append((f, j))
    out = []
    k = 0
    while k * STRIDE + FRAG <= len(image):
        for f, j in by_bytes.get(bytes(image[k * STRIDE:k * STRIDE + FRAG]), []):
            out.append((k, f, j))
        k += 1
    return sorted(out)


def as_list(arr) -> list:
    return [(int(a), int(b), int(c)) for a, b, c in zip(arr["disk_sector"], arr["file_id"], arr["file_sector"])]


def tricky_frag_case(seed: int):
    rng = np.random.default_rng(seed)
    rnd = lambda n: rng.integers(0, 256, n, dtype=np.uint8)
    shared = rnd(FRAG)
    a = rnd(5 * FRAG + 17)                      # partial tail fragment
    a[FRAG:2 * FRAG] = 0                        # all-zero fragment: excluded
    a[3 * FRAG:4 * FRAG] = 0x77                 # one-byte fill: excluded
    a[4 * FRAG:5 * FRAG] = shared
    b = np.concatenate([shared, rnd(2 * FRAG), shared])  # shared across files and repeated
    c = rnd(FRAG - 1)                           # no whole fragment
    d = np.zeros(FRAG, np.uint8)
    d[63] = 9                                   # all zero but one byte: kept
    files = [a, b, c, d, np.zeros(0, np.uint8)]
    pieces = []
    for _ in range(30):
        r = int(rng.integers(0, 7))
        if r == 0:
            pieces.append(rnd(int(rng.integers(1, 9)) * STRIDE))     # shift by a multiple of 4
        elif r == 1:
            pieces.append(a[: int(rng.integers(1, a.size))])         # a prefix of a file
        elif r == 2:
            pieces.append(b)
        elif r == 3:
            pieces.append(d)
        elif r == 4:
            pieces.append(np.zeros(int(rng.integers(1, 200)), np.uint8))
        elif r == 5:
            pieces.append(np.full(FRAG + 8, 0x77, np.uint8))          # holds a whole window of a fill
        else:
            pieces.append(rnd(int(rng.integers(1, 100))))            # any length: off the 4-byte grid too
    image = np.concatenate(pieces + [b[:FRAG + 3]])
    return image, files


@pytest.mark.parametrize("seed", range(10))
def test_frag_routes_equal_definition(seed):
    image, files = tricky_frag_case(seed)
    want = py_frag_match(image.tobytes(), [f.tobytes() for f in files])
    assert as_list(oracle.frag_match_brute(image, files)) == want
    assert as_list(oracle.frag_match(image, files)) == want


def test_frag_window_bounds_and_short_images():
    x = np.random.default_rng(1).integers(0, 256, FRAG, dtype=np.uint8)
    for pad in range(0, 9):
        img = np.concatenate([np.zeros(pad * STRIDE, np.uint8), x])  # ends exactly at the image end
        got = as_list(oracle.frag_match(img, [x]))
        assert got == [(pad, 0, 0)]
        assert as_list(oracle.frag_match(img[:-1], [x])) == []         # one byte short
    for n in range(0, FRAG):
        assert oracle.frag_match(x[:n], [x]).size == 0
    # a window off the 4-byte grid is not a window
    img = np.concatenate([np.zeros(2, np.uint8), x, np.zeros(6, np.uint8)])
    assert oracle.frag_match(img, [x]).size == 0


def test_frag_every_offset_residue():
    """A planted file found at every 4-byte offset modulo 64: window k = o/4 + 16 j."""
    rng = np.random.default_rng(2)
    logo = rng.integers(0, 256, 3 * FRAG, dtype=np.uint8)
    for o in range(0, 2 * FRAG, STRIDE):
        img = np.concatenate([rng.integers(0, 256, o, dtype=np.uint8), logo, rng.integers(0, 256, 50, dtype=np.uint8)])
        got = as_list(oracle.frag_match(img, [logo]))
        assert got == [(o // STRIDE + 16 * j, 0, j) for j in range(3)], o


def test_fragment_trivial_rule():
    assert oracle.fragment_trivial(np.zeros(FRAG, np.uint8))
    assert oracle.fragment_trivial(np.full(FRAG, 0xFF, np.uint8))
    for pos in (0, 1, 63):
        s = np.zeros(FRAG, np.uint8)
        s[pos] = 1
        assert not oracle.fragment_trivial(s)


def test_frag_plant_log():
    for seed in range(3):
        fp = synth.frag_config(f"frag_small:{(1 << 20) + 7 * seed}:24:{seed + 40}")
        img = fp.image_host()
        logos = fp.logos()
        got = oracle.frag_match(img, logos)
        exp = fp.expected_planted()
        assert exp.size > 100
        gs = set(as_list(got))
        assert set(as_list(exp)) <= gs
        # every extra triple is a fragment shared with a planted one (a common header)
        for k, f, j in gs - set(as_list(exp)):
            w = img[k * STRIDE:k * STRIDE + FRAG]
            assert np.array_equal(w, logos[f][j * FRAG:(j + 1) * FRAG])
            assert fp.header_len[f] > 0


def test_frag_brute_on_generated():
    fp = synth.frag_config("frag_small:600000:6:9")
    img = fp.image_host()
    logos = fp.logos()
    assert np.array_equal(oracle.frag_match(img, logos), oracle.frag_match_brute(img, logos))
