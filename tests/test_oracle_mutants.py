"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/oracle.c`` (a dropped term, a wrong index, a
wrong constant, a wrong comparison), builds that copy on the CPU, and checks that at least one
pin of tests/test_oracle.py fails against it. The real oracle is never modified.
"""
import ctypes
import hashlib
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from test_oracle import as_list, py_match, tricky_case
from test_oracle_fragments import py_frag_match, tricky_frag_case

MUTANTS = {
    "rotation amount": ("{7, 12, 17, 22}", "{7, 12, 17, 21}"),
    "round-2 message index": ("(1 + 5 * j) % 16", "(5 * j) % 16"),
    "round-3 message index": ("(5 + 3 * j) % 16", "(3 + 5 * j) % 16"),
    "round-3 function": ("return x ^ y ^ z;", "return x ^ y ^ ~z;"),
    "round-4 function": ("return y ^ (x | ~z);", "return y ^ (x | z);"),
    "MD5 F function (first 16 operations)": ("return (x & y) | (~x & z);", "return (x & y) | (x & z);"),
    "sine index": ("T_sine[i + 1]", "T_sine[i]"),
    "sine scale": ("4294967296.0 * fabs", "4294967295.0 * fabs"),
    "padding boundary": ("(rem < 56) ? 64 : 128", "(rem <= 56) ? 64 : 128"),
    "length in bytes not bits": ("uint64_t bits = len * 8u;", "uint64_t bits = len;"),
    "feed-forward dropped": ("st[3] += d;", "st[3] = d;"),
    "register roles": ("c = b;\n    b = t;", "c = t;\n    b = b;"),
    "big-endian words": ("(uint32_t)blk[4 * j] | ((uint32_t)blk[4 * j + 1] << 8)",
                         "(uint32_t)blk[4 * j + 1] | ((uint32_t)blk[4 * j] << 8)"),
    "initial state": ("0x10325476u}; /* Section 3.3 */", "0x10325477u}; /* Section 3.3 */"),
    "trivial rule only zero": ("if (sector[j] != sector[0]) return 0;", "if (sector[j] != 0) return 0;"),
    "trivial rule off": ("for (uint32_t j = 1; j < SECTOR; j++)\n    if (sector[j] != sector[0]) return 0;\n  return 1;",
                         "return 0;"),
    "first equal digest only": ("while (b < db->n && memcmp(db->e[b].digest, dg, 16) == 0) b++;",
                                "if (b < db->n && memcmp(db->e[b].digest, dg, 16) == 0) b++;"),
    "sort by file descending": ("if (a->file_id != b->file_id) return a->file_id < b->file_id ? -1 : 1;\n  if (a->file_sector != b->file_sector) return a->file_sector < b->file_sector ? -1 : 1;\n  return 0;\n}\n\n/* ------------------------------------------------------------- brute",
                                "if (a->file_id != b->file_id) return a->file_id > b->file_id ? -1 : 1;\n  if (a->file_sector != b->file_sector) return a->file_sector < b->file_sector ? -1 : 1;\n  return 0;\n}\n\n/* ------------------------------------------------------------- brute"),
    "window offset dropped": ("out[n].disk_sector = first_index + i;", "out[n].disk_sector = i;"),
    "last master sector dropped": ("uint64_t n_fs = file_bytes[f] / SECTOR;\n    for (uint64_t s = 0; s < n_fs; s++) {\n      const uint8_t* m = files[f] + s * SECTOR;\n      if (oracle_sector_trivial(m)) continue;\n      db",
                                   "uint64_t n_fs = file_bytes[f] / SECTOR;\n    if (n_fs) n_fs--;\n    for (uint64_t s = 0; s < n_fs; s++) {\n      const uint8_t* m = files[f] + s * SECTOR;\n      if (oracle_sector_trivial(m)) continue;\n      db"),
    "djb2 multiplier": ("h = h * 33u + msg[i];", "h = h * 31u + msg[i];"),
    "djb2 initial value": ("uint64_t h = 5381u;", "uint64_t h = 5380u;"),
    "crc polynomial": ("const uint64_t low = 0x1Bu;", "const uint64_t low = 0x1Au;"),
    "crc bit order": ("for (int b = 7; b >= 0; b--) {", "for (int b = 0; b <= 7; b++) {"),
    "crc without the x^64 factor": ("for (int b = 0; b < 64; b++) {\n    const uint64_t top = rem >> 63;\n    rem <<= 1;",
                                    "for (int b = 0; b < 0; b++) {\n    const uint64_t top = rem >> 63;\n    rem <<= 1;"),
    "weak signatures not confirmed": ("const int confirm = db->sig == SIG_DJB2_64 || db->sig == SIG_CRC64;",
                                      "const int confirm = 0;"),
    "position base added not subtracted": ("((all[k].disk_sector % 8u) + 8u - (base_offset % 8u)) % 8u",
                                           "((all[k].disk_sector % 8u) + (base_offset % 8u)) % 8u"),
    "position from the disk sector only": ("if (tau_disk != all[k].file_sector % 8u) continue;",
                                           "if (tau_disk != 0u) continue;"),
    "fragment window stride": ("#define FRAG_STRIDE 4u", "#define FRAG_STRIDE 8u"),
    "fragment last window dropped": ("(image_bytes - FRAG) / FRAG_STRIDE + 1", "(image_bytes - FRAG) / FRAG_STRIDE"),
    "fragment rule only zero": ("if (frag[j] != frag[0]) return 0;", "if (frag[j] != 0) return 0;"),
    "fragment master stride": ("const uint8_t* b = files[f] + j * FRAG;", "const uint8_t* b = files[f] + j * FRAG_STRIDE;"),
    "no-pad state after 7 blocks": ("for (int b = 0; b < 8; b++) md5_block(st, sector + 64 * b);",
                                    "for (int b = 0; b < 7; b++) md5_block(st, sector + 64 * b);"),
}


def _build_mutant(src: str, old: str, new: str, td: str) -> str:
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    path = os.path.join(td, "m.c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    lib = os.path.join(td, "libm.so")
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-std=c11", path, "-o", lib, "-lm"], check=True,
                   capture_output=True)
    return lib


def _signature_pins_pass() -> bool:
    """The pins of tests/test_oracle_signatures.py, condensed."""
    import test_oracle_signatures as ts

    rng = np.random.default_rng(6)
    x = rng.integers(40, 200, 512, dtype=np.uint8)
    if oracle.md5_finish_sector(oracle.md5_nopad(x)) != hashlib.md5(x.tobytes()).digest():
        return False
    if oracle.djb2_64(b"") != 5381 or oracle.djb2_64(np.zeros(512, np.uint8)) != (5381 * pow(33, 512, 1 << 64)) & ts.M64:
        return False
    msg = bytearray(16)
    msg[3] = 2
    if oracle.crc64(bytes(msg)) != ts.x_pow_mod(8 * 12 + 1 + 64, ts.GEN):
        return False
    if oracle.crc64(x) != ts.poly_mod(int.from_bytes(x.tobytes(), "big") << 64, ts.GEN):
        return False
    image, files = tricky_case(1)
    m = files[0][2 * 512:3 * 512]
    m[:] = x
    image = np.concatenate([image[: image.size // 512 * 512], ts.djb2_collision(x, 10), ts.crc_collision(x, 99), x])
    want = py_match(image.tobytes(), [f.tobytes() for f in files])
    return all(as_list(oracle.match_sig(image, files, sig)) == want for sig in (1, 2, 3))


def _position_pins_pass() -> bool:
    """The position-keyed pin: the definition's triples filtered by cluster position."""
    image, files = tricky_case(2)
    full = py_match(image.tobytes(), [f.tobytes() for f in files])
    for base in (0, 3, 13):
        want = [t for t in full if (t[0] - base) % 8 == t[2] % 8]
        if as_list(oracle.match_position(image, files, base)) != want:
            return False
    return True


def _fragment_pins_pass() -> bool:
    """The fragment pins: both routes against the Python definition on the tricky inputs."""
    for seed in range(3):
        image, files = tricky_frag_case(seed)
        want = py_frag_match(image.tobytes(), [f.tobytes() for f in files])
        if as_list(oracle.frag_match_brute(image, files)) != want or as_list(oracle.frag_match(image, files)) != want:
            return False
    x = np.random.default_rng(1).integers(0, 256, 64, dtype=np.uint8)
    img = np.concatenate([np.zeros(12, np.uint8), x])  # the last window ends at the image end
    return as_list(oracle.frag_match(img, [x])) == [(3, 0, 0)] == as_list(oracle.frag_match_brute(img, [x]))


def _pins_pass() -> bool:
    """The pins of tests/test_oracle.py, condensed; False as soon as one fails."""
    if not _signature_pins_pass() or not _position_pins_pass() or not _fragment_pins_pass():
        return False
    rng = np.random.default_rng(5)
    for length in (0, 1, 55, 56, 63, 64, 100, 512, 1000):
        d = rng.integers(0, 256, length, dtype=np.uint8).tobytes()
        if oracle.md5(d) != hashlib.md5(d).digest():
            return False
    for seed in range(4):
        image, files = tricky_case(seed)
        want = py_match(image.tobytes(), [f.tobytes() for f in files])
        if as_list(oracle.match_brute(image, files)) != want:
            return False
        if as_list(oracle.match_hash(image, files)) != want:
            return False
        db = oracle.OracleDB(files)
        part = as_list(db.lookup(image[3 * 512:20 * 512], 3))
        db.close()
        if part != [t for t in want if 3 <= t[0] < 20]:
            return False
    return True


def test_real_oracle_passes_condensed_pins():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    with open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")) as fh:
        src = fh.read()
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as td:
        lib = oracle.bind(ctypes.CDLL(_build_mutant(src, old, new, td)))
        monkeypatch.setattr(oracle, "_lib", lib)
        assert not _pins_pass(), f"mutant '{name}' passed every pin"
