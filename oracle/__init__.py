"""CPU oracle for sector-signature data carving (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package. The product path (the CUDA library and ``paper_0901_1307_gb300``) never does, and
this package imports nothing from it.

The arithmetic lives in ``oracle.c`` (plain C, built with gcc, optionally OpenMP-parallel over
independent sectors). This module only marshals numpy arrays in and out.

Functions and the passages they follow:

* ``md5(data)`` -- RFC 1321 MD5 of a byte string (the signature the paper's Section 2.1 proposes).
* ``md5_sectors(arr)`` -- MD5 of every 512-byte sector of an array.
* ``sector_trivial(sector)`` -- the exclusion rule: all 512 bytes equal.
* ``match_brute(image, files)`` -- the result by its definition (Section 1, Section 3.1: a disk
  sector matches a master sector when they are byte-for-byte equal): every (disk_sector, file_id,
  file_sector), sorted.
* ``match_hash(image, files)`` / ``OracleDB`` -- the method's route (Section 3.1): signatures of the
  kept master sectors, each disk sector's signature looked up, equal signatures reported, sorted.
* ``match_sig(image, files, sig)`` -- the same with another signature: MD5 without padding, djb2-64
  (Eq. 1) or CRC64 (Section 2.1); candidates of the 64-bit ones are confirmed byte for byte.
* ``signature`` / ``signatures(data, sig)`` -- one sector's (every sector's) signature under any kind;
  ``window_signatures(image, sig)`` -- every 64-byte window's at a 4-byte offset (Section 5);
  ``md5_blocks`` -- the MD5 state after whole blocks without padding.

Parity pins (tests/test_oracle.py): MD5 against hashlib (OpenSSL) and md5sum; ``match_hash``
against ``match_brute`` on tiny inputs with duplicates, fills and partial sectors; both against
the generator's plant log.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SECTOR = 512
TRIPLE_DTYPE = np.dtype([("disk_sector", "<u8"), ("file_id", "<u4"), ("file_sector", "<u4")])


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def bind(lib):
    """Declare the C signatures on a loaded oracle library (also used to load test variants)."""
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    lib.oracle_md5.argtypes = [vp, u64, vp]
    lib.oracle_md5.restype = None
    lib.oracle_md5_sectors.argtypes = [vp, u64, vp]
    lib.oracle_md5_sectors.restype = None
    lib.oracle_sector_trivial.argtypes = [vp]
    lib.oracle_sector_trivial.restype = ctypes.c_int
    sig = [vp, u64, vp, vp, u32, vp, u64]
    lib.oracle_match_brute.argtypes = sig
    lib.oracle_match_brute.restype = ctypes.c_int64
    lib.oracle_match_hash.argtypes = sig
    lib.oracle_match_hash.restype = ctypes.c_int64
    lib.oracle_db_build.argtypes = [vp, vp, u32]
    lib.oracle_db_build.restype = vp
    lib.oracle_db_size.argtypes = [vp]
    lib.oracle_db_size.restype = u64
    lib.oracle_db_free.argtypes = [vp]
    lib.oracle_db_free.restype = None
    lib.oracle_db_lookup.argtypes = [vp, vp, u64, u64, vp, u64]
    lib.oracle_db_lookup.restype = ctypes.c_int64
    lib.oracle_md5_nopad.argtypes = [vp, vp]
    lib.oracle_md5_nopad.restype = None
    lib.oracle_md5_finish_sector.argtypes = [vp, vp]
    lib.oracle_md5_finish_sector.restype = None
    lib.oracle_djb2_64.argtypes = [vp, u64]
    lib.oracle_djb2_64.restype = u64
    lib.oracle_crc64.argtypes = [vp, u64]
    lib.oracle_crc64.restype = u64
    lib.oracle_signature.argtypes = [vp, ctypes.c_int, vp]
    lib.oracle_signature.restype = None
    lib.oracle_match_sig.argtypes = [vp, u64, vp, vp, u32, ctypes.c_int, vp, u64]
    lib.oracle_match_sig.restype = ctypes.c_int64
    lib.oracle_frag_match_brute.argtypes = [vp, u64, vp, vp, u32, vp, u64]
    lib.oracle_frag_match_brute.restype = ctypes.c_int64
    lib.oracle_frag_match.argtypes = [vp, u64, vp, vp, u32, vp, u64]
    lib.oracle_frag_match.restype = ctypes.c_int64
    lib.oracle_fragment_trivial.argtypes = [vp]
    lib.oracle_fragment_trivial.restype = ctypes.c_int
    lib.oracle_match_position.argtypes = [vp, u64, vp, vp, u32, u64, vp, u64]
    lib.oracle_match_position.restype = ctypes.c_int64
    lib.oracle_db_build_sig.argtypes = [vp, vp, u32, ctypes.c_int]
    lib.oracle_db_build_sig.restype = vp
    lib.oracle_signatures.argtypes = [vp, u64, ctypes.c_int, vp]
    lib.oracle_signatures.restype = None
    lib.oracle_md5_blocks.argtypes = [vp, u64, vp]
    lib.oracle_md5_blocks.restype = None
    lib.oracle_window_signatures.argtypes = [vp, u64, ctypes.c_int, vp]
    lib.oracle_window_signatures.restype = None
    lib.oracle_threads.argtypes = []
    lib.oracle_threads.restype = ctypes.c_int
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build()))
        return _lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        a = np.frombuffer(bytes(a), dtype=np.uint8)
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint8:
        a = a.view(np.uint8)
    return a.reshape(-1)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return _load().oracle_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def md5(data) -> bytes:
    """RFC 1321 MD5 digest (16 bytes) of ``data``."""
    a = _u8(data)
    out = np.zeros(16, np.uint8)
    _load().oracle_md5(_ptr(a), a.size, out.ctypes.data)
    return out.tobytes()


def md5_sectors(data) -> np.ndarray:
    """MD5 of every whole 512-byte sector of ``data``: uint8 array of shape (n, 16)."""
    a = _u8(data)
    n = a.size // SECTOR
    out = np.zeros((n, 16), np.uint8)
    if n:
        _load().oracle_md5_sectors(_ptr(a), n, out.ctypes.data)
    return out


def sector_trivial(sector) -> bool:
    a = _u8(sector)
    assert a.size == SECTOR
    return bool(_load().oracle_sector_trivial(_ptr(a)))


class _Files:
    """Keeps the file arrays alive and exposes (const uint8_t**, const uint64_t*)."""

    def __init__(self, files):
        self.arrs = [_u8(f) for f in files]
        n = len(self.arrs)
        self.ptrs = (ctypes.c_void_p * max(n, 1))(*[_ptr(a) or None for a in self.arrs])
        self.sizes = (ctypes.c_uint64 * max(n, 1))(*[a.size for a in self.arrs])
        self.n = n


def _run_match(fn, image, files) -> np.ndarray:
    img = _u8(image)
    fl = _Files(files)
    cap = 1 << 16
    while True:
        out = np.zeros(cap, TRIPLE_DTYPE)
        n = fn(_ptr(img), img.size, fl.ptrs, fl.sizes, fl.n, out.ctypes.data, cap)
        if n < 0:
            raise MemoryError("oracle: allocation failed")
        if n <= cap:
            return out[:n].copy()
        cap = int(n)


def match_brute(image, files) -> np.ndarray:
    """All (disk_sector, file_id, file_sector) with byte-equal sectors, by exhaustive memcmp."""
    return _run_match(_load().oracle_match_brute, image, files)


SIG_MD5, SIG_MD5_NOPAD, SIG_DJB2_64, SIG_CRC64 = 0, 1, 2, 3


def md5_nopad(sector) -> bytes:
    """MD5 state after the 8 data blocks of a 512-byte sector (no padding block)."""
    a = _u8(sector)
    assert a.size == SECTOR
    out = np.zeros(16, np.uint8)
    _load().oracle_md5_nopad(_ptr(a), out.ctypes.data)
    return out.tobytes()


def md5_finish_sector(state: bytes) -> bytes:
    a = _u8(state)
    out = np.zeros(16, np.uint8)
    _load().oracle_md5_finish_sector(_ptr(a), out.ctypes.data)
    return out.tobytes()


def djb2_64(data) -> int:
    a = _u8(data)
    return int(_load().oracle_djb2_64(_ptr(a), a.size))


def crc64(data) -> int:
    a = _u8(data)
    return int(_load().oracle_crc64(_ptr(a), a.size))


def signature(sector, sig: int) -> bytes:
    a = _u8(sector)
    assert a.size == SECTOR
    out = np.zeros(16, np.uint8)
    _load().oracle_signature(_ptr(a), sig, out.ctypes.data)
    return out.tobytes()


def signatures(data, sig: int) -> np.ndarray:
    """``signature`` of every whole 512-byte sector of data: an (n, 16) uint8 array."""
    a = _u8(data)
    n = a.size // SECTOR
    out = np.zeros((n, 16), np.uint8)
    if n:
        _load().oracle_signatures(_ptr(a), n, int(sig), out.ctypes.data)
    return out


def md5_blocks(data) -> bytes:
    """MD5 state after the whole 64-byte blocks of data, without a padding block."""
    a = _u8(data)
    out = np.zeros(16, np.uint8)
    _load().oracle_md5_blocks(_ptr(a), a.size // 64, out.ctypes.data)
    return out.tobytes()


def window_signatures(image, sig: int) -> np.ndarray:
    """The signature of every 64-byte window at a 4-byte offset (Section 5): (n_windows, 16)
    uint8; djb2-64 little-endian in the first 8 bytes."""
    a = _u8(image)
    n = (a.size - 64) // 4 + 1 if a.size >= 64 else 0
    out = np.zeros((n, 16), np.uint8)
    if n:
        _load().oracle_window_signatures(_ptr(a), a.size, int(sig), out.ctypes.data)
    return out


def match_sig(image, files, sig: int) -> np.ndarray:
    """The method with a chosen signature (64-bit ones confirmed byte for byte)."""
    lib = _load()
    return _run_match(lambda *a: lib.oracle_match_sig(*a[:5], sig, *a[5:]), image, files)


def match_position(image, files, base_offset: int = 0) -> np.ndarray:
    """Position-keyed matching (tables S_tau): triples whose disk sector has the master sector's
    position in its 8-sector cluster, disk clusters counted from sector base_offset."""
    lib = _load()
    return _run_match(lambda *a: lib.oracle_match_position(*a[:5], int(base_offset), *a[5:]), image, files)


FRAG, FRAG_STRIDE = 64, 4


def frag_match_brute(image, files) -> np.ndarray:
    """Fragments (Section 5): every (window k, file f, fragment j) with image bytes
    [4k, 4k+64) equal to bytes [64j, 64j+64) of file f (kept fragments only), by exhaustive
    memcmp. The window index is in the disk_sector field, j in file_sector."""
    return _run_match(_load().oracle_frag_match_brute, image, files)


def frag_match(image, files) -> np.ndarray:
    """The fragment result through the kept fragments sorted by their bytes and a binary
    search per window."""
    return _run_match(_load().oracle_frag_match, image, files)


def fragment_trivial(frag) -> bool:
    a = _u8(frag)
    assert a.size == FRAG
    return bool(_load().oracle_fragment_trivial(_ptr(a)))


def match_hash(image, files) -> np.ndarray:
    """The same result reached through MD5 signatures and a sorted signature database."""
    return _run_match(_load().oracle_match_hash, image, files)


class OracleDB:
    """The signature database of a master set, for looking up any subset of disk sectors."""

    def __init__(self, files, sig: int = 0):
        fl = _Files(files)
        self._files = fl  # borrowed by the database
        lib = _load()
        self._h = lib.oracle_db_build_sig(fl.ptrs, fl.sizes, fl.n, sig)
        if not self._h:
            raise MemoryError("oracle: database allocation failed")

    def __len__(self) -> int:
        return int(_load().oracle_db_size(self._h))

    def lookup(self, sectors, first_index: int = 0) -> np.ndarray:
        """Triples for consecutive sectors whose first one is disk sector ``first_index``."""
        a = _u8(sectors)
        n = a.size // SECTOR
        cap = max(16, n)
        while True:
            out = np.zeros(cap, TRIPLE_DTYPE)
            k = _load().oracle_db_lookup(self._h, _ptr(a), n, int(first_index), out.ctypes.data, cap)
            if k < 0:
                raise MemoryError("oracle: lookup allocation failed")
            if k <= cap:
                return out[:k].copy()
            cap = int(k)

    def close(self) -> None:
        if getattr(self, "_h", None):
            _load().oracle_db_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
