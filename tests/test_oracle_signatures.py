"""Pins for the oracle's other sector signatures (no GPU): MD5 without the padding block,
djb2 with a 64-bit accumulator (Eq. 1) and CRC64 with generator x^64 + x^4 + x^3 + x + 1. Each is
checked against mathematics that does not re-type its own code: hashlib (through the padding
block), closed forms of Eq. 1, GF(2) polynomial arithmetic for the CRC, and, for the matchers,
the byte-equality definition on inputs that hold real signature collisions."""
import hashlib

import numpy as np
import pytest

import oracle
from test_oracle import as_list, py_match, tricky_case

SECTOR = 512
M64 = (1 << 64) - 1
GEN = (1 << 64) | 0x1B  # x^64 + x^4 + x^3 + x + 1


def test_md5_nopad_then_padding_block_is_md5():
    rng = np.random.default_rng(2)
    for k in range(40):
        x = rng.integers(0, 256, SECTOR, dtype=np.uint8)
        if k == 1:
            x[:] = 0
        if k == 2:
            x[:] = 0xA5
        st = oracle.md5_nopad(x)
        assert oracle.md5_finish_sector(st) == hashlib.md5(x.tobytes()).digest()
        assert st != hashlib.md5(x.tobytes()).digest()
        assert oracle.signature(x, oracle.SIG_MD5_NOPAD) == st
        assert oracle.signature(x, oracle.SIG_MD5) == hashlib.md5(x.tobytes()).digest()


def test_djb2_closed_forms():
    assert oracle.djb2_64(b"") == 5381
    for b in (0, 1, 97, 255):
        assert oracle.djb2_64(bytes([b])) == (5381 * 33 + b) & M64
    zero = np.zeros(SECTOR, np.uint8)
    assert oracle.djb2_64(zero) == (5381 * pow(33, SECTOR, 1 << 64)) & M64
    # every byte contributes s_i * 33^(n-1-i): perturbing one byte moves the hash by that term
    rng = np.random.default_rng(3)
    x = rng.integers(0, 200, SECTOR, dtype=np.uint8)
    h = oracle.djb2_64(x)
    for i in (0, 1, 100, 510, 511):
        y = x.copy()
        y[i] += 7
        assert (oracle.djb2_64(y) - h) & M64 == (7 * pow(33, SECTOR - 1 - i, 1 << 64)) & M64


def poly_mod(a: int, m: int) -> int:
    """Remainder of the GF(2) polynomial a modulo m (bit k = coefficient of x^k)."""
    dm = m.bit_length() - 1
    while a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def x_pow_mod(k: int, m: int) -> int:
    """x^k mod m by square-and-multiply in GF(2)[x]."""
    def mul(a, b):
        r = 0
        while b:
            if b & 1:
                r ^= a
            a <<= 1
            b >>= 1
        return poly_mod(r, m)

    result, base = 1, poly_mod(2, m)
    while k:
        if k & 1:
            result = mul(result, base)
        base = mul(base, base)
        k >>= 1
    return result


def test_crc64_single_bits_are_powers_of_x():
    # message bit j of byte i (MSB first) is the coefficient of x^(8(n-1-i) + j) in M(x); its CRC
    # is x^(that + 64) mod G
    n = 16
    for i in (0, 3, 15):
        for j in (0, 1, 7):
            msg = bytearray(n)
            msg[i] = 1 << j
            assert oracle.crc64(bytes(msg)) == x_pow_mod(8 * (n - 1 - i) + j + 64, GEN)


def test_crc64_linear_and_residue():
    rng = np.random.default_rng(4)
    a = rng.integers(0, 256, SECTOR, dtype=np.uint8)
    b = rng.integers(0, 256, SECTOR, dtype=np.uint8)
    assert oracle.crc64(a ^ b) == oracle.crc64(a) ^ oracle.crc64(b)
    assert oracle.crc64(np.zeros(SECTOR, np.uint8)) == 0
    c = oracle.crc64(a)
    # appending the remainder (most significant byte first) leaves remainder 0
    assert oracle.crc64(a.tobytes() + c.to_bytes(8, "big")) == 0
    # the remainder of the message polynomial itself, computed independently
    m = int.from_bytes(a.tobytes(), "big")
    assert c == poly_mod(m << 64, GEN)


def djb2_collision(x: np.ndarray, i: int) -> np.ndarray:
    """A different sector with the same djb2-64: +1 at byte i and -33 at byte i+1 cancel."""
    y = x.copy()
    assert y[i] < 255 and y[i + 1] >= 33
    y[i] += 1
    y[i + 1] -= 33
    return y


def crc_collision(x: np.ndarray, bit: int) -> np.ndarray:
    """A different sector with the same CRC64: XOR with the generator shifted by `bit`."""
    m = int.from_bytes(x.tobytes(), "big") ^ (GEN << bit)
    return np.frombuffer(m.to_bytes(SECTOR, "big"), np.uint8).copy()


def _mulmod(a: int, b: int) -> int:
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a >> 64:
            a ^= GEN
    return r


def crc_high_twin(x: np.ndarray, k: int) -> np.ndarray:
    """A sector whose CRC64 equals x's XOR (k << 32): XOR x with E = k(x) x^32 x^-64 mod G, so the
    low 32 bits (the table's first key word) agree and the high ones differ."""
    inv_x = (1 << 63) | 0b1101  # x (x^63 + x^3 + x^2 + 1) = 1 mod G
    e = k
    for _ in range(32):
        e = _mulmod(e, inv_x)
    m = int.from_bytes(x.tobytes(), "big") ^ e
    return np.frombuffer(m.to_bytes(SECTOR, "big"), np.uint8).copy()


def test_crc_high_twin_construction():
    x = np.random.default_rng(3).integers(0, 256, SECTOR, dtype=np.uint8)
    for k in (1, 2, 0xDEAD):
        y = crc_high_twin(x, k)
        assert poly_mod(int.from_bytes(y.tobytes(), "big") << 64, GEN) == \
            poly_mod(int.from_bytes(x.tobytes(), "big") << 64, GEN) ^ (k << 32)
        assert oracle.crc64(y) == oracle.crc64(x) ^ (k << 32)


def test_constructed_collisions_collide():
    rng = np.random.default_rng(5)
    x = rng.integers(40, 200, SECTOR, dtype=np.uint8)
    y = djb2_collision(x, 100)
    assert oracle.djb2_64(x) == oracle.djb2_64(y) and not np.array_equal(x, y)
    z = crc_collision(x, 777)
    assert oracle.crc64(x) == oracle.crc64(z) and not np.array_equal(x, z)


@pytest.mark.parametrize("sig", [0, 1, 2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_match_sig_equals_definition(sig, seed):
    image, files = tricky_case(seed)
    # add sectors that collide with master sectors under djb2 and CRC64 but differ in bytes
    rng = np.random.default_rng(seed + 100)
    m = files[0][2 * SECTOR:3 * SECTOR].copy()
    m[:] = rng.integers(40, 200, SECTOR, dtype=np.uint8)
    files[0][2 * SECTOR:3 * SECTOR] = m
    image = np.concatenate([image[: image.size // SECTOR * SECTOR], djb2_collision(m, 10), crc_collision(m, 99), m])
    want = py_match(image.tobytes(), [f.tobytes() for f in files])
    assert as_list(oracle.match_sig(image, files, sig)) == want


def test_batch_signatures_equal_single_ones():
    rng = np.random.default_rng(21)
    data = rng.integers(0, 256, SECTOR * 37, dtype=np.uint8)
    data[SECTOR * 3: SECTOR * 4] = 0
    data[SECTOR * 5: SECTOR * 6] = 0x41
    for sig in (oracle.SIG_MD5, oracle.SIG_MD5_NOPAD, oracle.SIG_DJB2_64, oracle.SIG_CRC64):
        got = oracle.signatures(np.concatenate([data, data[:100]]), sig)  # a partial tail is ignored
        assert got.shape == (37, 16)
        for i in range(37):
            assert got[i].tobytes() == oracle.signature(data[SECTOR * i: SECTOR * (i + 1)], sig)


def test_md5_blocks_then_rfc_padding_is_md5():
    # the RFC's padding for a 64-byte message: 0x80, zeros, then the bit length 512 as a 64-bit
    # little-endian integer, all in one more block
    pad = np.zeros(64, np.uint8)
    pad[0] = 0x80
    pad[56:64] = np.frombuffer((512).to_bytes(8, "little"), np.uint8)
    rng = np.random.default_rng(22)
    for _ in range(30):
        w = rng.integers(0, 256, 64, dtype=np.uint8)
        assert oracle.md5_blocks(np.concatenate([w, pad])) == hashlib.md5(w.tobytes()).digest()
        assert oracle.md5_blocks(w) != hashlib.md5(w.tobytes()).digest()
    x = rng.integers(0, 256, SECTOR, dtype=np.uint8)
    assert oracle.md5_blocks(x) == oracle.md5_nopad(x)


def _djb2_py(b: bytes) -> int:
    h = 5381
    for c in b:
        h = (h * 33 + c) & M64
    return h


def test_window_signatures_follow_their_definitions():
    rng = np.random.default_rng(23)
    img = rng.integers(0, 256, 64 * 5 + 23, dtype=np.uint8)  # windows do not end on the grid
    img[100:180] = 0
    n_win = (img.size - 64) // 4 + 1
    md5 = oracle.window_signatures(img, oracle.SIG_MD5)
    nop = oracle.window_signatures(img, oracle.SIG_MD5_NOPAD)
    djb = oracle.window_signatures(img, oracle.SIG_DJB2_64)
    assert md5.shape == nop.shape == djb.shape == (n_win, 16)
    for k in range(n_win):
        w = img[4 * k: 4 * k + 64].tobytes()
        assert md5[k].tobytes() == hashlib.md5(w).digest()
        assert nop[k].tobytes() == oracle.md5_blocks(np.frombuffer(w, np.uint8))
        assert djb[k].tobytes() == _djb2_py(w).to_bytes(8, "little") + bytes(8)
    assert oracle.window_signatures(img[:63], oracle.SIG_MD5).shape == (0, 16)
    assert oracle.window_signatures(img[:64], oracle.SIG_DJB2_64).shape == (1, 16)
