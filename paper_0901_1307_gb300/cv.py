"""Python binding of libcv.so (include/cv.h): argument marshalling only.

Every step of the scan runs in the library's CUDA kernels. There is no CPU path: if libcv.so is
missing or no CUDA device is usable, the calls raise.

Buffers can be given as torch tensors (CPU or CUDA), numpy arrays, bytes, or (pointer, n_bytes)
tuples; streams as torch.cuda.Stream objects or raw cudaStream_t integers (None = default).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcv.so")

CV_OK = 0
CV_EINVAL = -1
CV_ENOMEM = -2
CV_ECUDA = -3
CV_ETABLEFULL = -4
CV_ECORRUPT = -5
CV_ETIMEOUT = -6
CV_ENODEV = -7
CV_ERANGE = -8
CV_BLOOM_AUTO = 0xFFFFFFFF
CV_SIG_MD5, CV_SIG_MD5_NOPAD, CV_SIG_DJB2_64, CV_SIG_CRC64 = 0, 1, 2, 3
CV_KEEP_ON_DEVICE = 1
CV_POSITION_ANY, CV_POSITION_CLUSTER = 0, 1
CV_LAYOUT_HASH, CV_LAYOUT_SORTED, CV_LAYOUT_AUTO = 0, 1, 2
CV_UNIT_SECTOR, CV_UNIT_FRAGMENT = 0, 1
SECTOR = 512

MATCH_DTYPE = np.dtype([("disk_sector", "<u8"), ("file_id", "<u4"), ("file_sector", "<u4")])

EXPORTS = ("cv_master_build", "cv_master_get_info", "cv_scan", "cv_matches", "cv_scan_get_stats", "cv_free",
           "cv_strerror", "cv_last_cuda_error", "cv_sector_digests", "cv_kernel_config_count",
           "cv_kernel_config_name", "cv_scan_noalloc", "cv_batch_create", "cv_batch_run", "cv_batch_wait",
           "cv_batch_matches", "cv_batch_get_info", "cv_server_create", "cv_submit", "cv_poll",
           "cv_server_get_stats", "cv_int_peak", "cv_selftest_wait_timeout", "cv_master_save", "cv_master_load",
           "cv_probe_profile", "cv_sector_signatures", "cv_window_signatures")
CV_EAGAIN = -9
CV_EIO = -10
CV_BATCH_BLOOM_AUTO = 0
CV_BATCH_BLOOM_OFF = 1
CV_BATCH_BLOOM_ON = 2
CV_NOALLOC_MAX_SECTORS = 1 << 19


class CVError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code}), last CUDA error {last_cuda_error()}")


class cv_buf(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n_bytes", ctypes.c_uint64)]


class cv_master_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("max_load", ctypes.c_float),
                ("bloom_bits_per_key", ctypes.c_uint32), ("signature", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("position_mode", ctypes.c_uint32), ("layout", ctypes.c_uint32), ("unit", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class cv_scan_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("chunk_bytes", ctypes.c_uint64), ("kernel_config", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("base_offset", ctypes.c_uint64)]


class cv_master_info(ctypes.Structure):
    _fields_ = [("n_files", ctypes.c_uint32), ("position_mode", ctypes.c_uint32), ("n_sectors", ctypes.c_uint64),
                ("n_kept", ctypes.c_uint64), ("n_unique", ctypes.c_uint64), ("n_slots", ctypes.c_uint64),
                ("bloom_bytes", ctypes.c_uint64), ("max_probe", ctypes.c_uint32), ("signature", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64), ("layout", ctypes.c_uint32), ("unit", ctypes.c_uint32)]


class cv_scan_stats(ctypes.Structure):
    _fields_ = [("sectors", ctypes.c_uint64), ("matches", ctypes.c_uint64), ("hit_sectors", ctypes.c_uint64),
                ("kernel_ms", ctypes.c_float), ("total_ms", ctypes.c_float), ("kernel_launches", ctypes.c_uint32),
                ("kernel_config", ctypes.c_int32), ("confirm_rejected", ctypes.c_uint64)]


class cv_probe_stats(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("layout", ctypes.c_uint32), ("sectors", ctypes.c_uint64),
                ("bloom_passed", ctypes.c_uint64), ("slot_reads", ctypes.c_uint64), ("key_reads", ctypes.c_uint64),
                ("found", ctypes.c_uint64)]


class cv_batch_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("autotune", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("match_capacity", ctypes.c_uint64), ("kernel_config", ctypes.c_uint32), ("bloom", ctypes.c_uint32),
                ("tune_cache", ctypes.c_char_p), ("sorted_copy", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class cv_batch_info(ctypes.Structure):
    _fields_ = [("kernel_config", ctypes.c_int), ("config_name", ctypes.c_char_p), ("bloom", ctypes.c_uint32),
                ("tuned", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint32), ("tensor_maps", ctypes.c_uint32),
                ("segments", ctypes.c_uint32), ("layout", ctypes.c_uint32), ("sectors", ctypes.c_uint64),
                ("match_capacity", ctypes.c_uint64), ("scan_ms", ctypes.c_float)]


class cv_server_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("max_live", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("work_unit_bytes", ctypes.c_uint64), ("kernel_config", ctypes.c_uint32),
                ("copy_streams", ctypes.c_uint32), ("max_copy_bytes", ctypes.c_uint64)]


class cv_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("bytes_scanned", ctypes.c_uint64), ("iterations", ctypes.c_uint64), ("units", ctypes.c_uint64),
                ("peak_bytes_in_flight", ctypes.c_uint64), ("mean_live_per_iteration", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("wall_s", ctypes.c_double)]


class cv_int_peak_info(ctypes.Structure):
    _fields_ = [("alu_ops_per_s", ctypes.c_double), ("fma_ops_per_s", ctypes.c_double),
                ("mixed_ops_per_s", ctypes.c_double), ("sm_clock_mhz", ctypes.c_double), ("sms", ctypes.c_int),
                ("reserved", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libcv.so and declare its signatures. Raises if the library was not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_0901_1307_gb300.build.build()")
        lib = ctypes.CDLL(path)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        lib.cv_master_build.argtypes = [ctypes.POINTER(cv_buf), u32, ctypes.POINTER(cv_master_opts), ctypes.POINTER(vp)]
        lib.cv_master_build.restype = i32
        lib.cv_master_get_info.argtypes = [vp, ctypes.POINTER(cv_master_info)]
        lib.cv_master_get_info.restype = i32
        lib.cv_master_save.argtypes = [vp, ctypes.c_char_p]
        lib.cv_master_save.restype = i32
        lib.cv_master_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
        lib.cv_master_load.restype = i32
        lib.cv_scan.argtypes = [vp, ctypes.POINTER(cv_buf), u32, ctypes.POINTER(cv_scan_opts), ctypes.POINTER(vp)]
        lib.cv_scan.restype = i32
        lib.cv_matches.argtypes = [vp, u32, ctypes.POINTER(vp), ctypes.POINTER(u64)]
        lib.cv_matches.restype = i32
        lib.cv_scan_get_stats.argtypes = [vp, ctypes.POINTER(cv_scan_stats)]
        lib.cv_scan_get_stats.restype = i32
        lib.cv_free.argtypes = [vp]
        lib.cv_free.restype = None
        lib.cv_strerror.argtypes = [i32]
        lib.cv_strerror.restype = ctypes.c_char_p
        lib.cv_last_cuda_error.argtypes = []
        lib.cv_last_cuda_error.restype = i32
        lib.cv_sector_digests.argtypes = [vp, u64, vp, vp, vp]
        lib.cv_sector_digests.restype = i32
        lib.cv_sector_signatures.argtypes = [vp, u64, u32, vp, vp, vp]
        lib.cv_sector_signatures.restype = i32
        lib.cv_window_signatures.argtypes = [vp, u64, u32, vp, vp]
        lib.cv_window_signatures.restype = i32
        lib.cv_kernel_config_count.argtypes = []
        lib.cv_kernel_config_count.restype = i32
        lib.cv_kernel_config_name.argtypes = [i32]
        lib.cv_kernel_config_name.restype = ctypes.c_char_p
        lib.cv_scan_noalloc.argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(u64), vp]
        lib.cv_scan_noalloc.restype = i32
        lib.cv_batch_create.argtypes = [vp, ctypes.POINTER(cv_buf), u32, ctypes.POINTER(cv_batch_opts),
                                        ctypes.POINTER(vp)]
        lib.cv_batch_create.restype = i32
        lib.cv_batch_run.argtypes = [vp, vp]
        lib.cv_batch_run.restype = i32
        lib.cv_batch_wait.argtypes = [vp, ctypes.POINTER(u64)]
        lib.cv_batch_wait.restype = i32
        lib.cv_batch_matches.argtypes = [vp, u32, ctypes.POINTER(vp), ctypes.POINTER(u64)]
        lib.cv_batch_matches.restype = i32
        lib.cv_batch_get_info.argtypes = [vp, ctypes.POINTER(cv_batch_info)]
        lib.cv_batch_get_info.restype = i32
        lib.cv_server_create.argtypes = [vp, ctypes.POINTER(cv_server_opts), ctypes.POINTER(vp)]
        lib.cv_server_create.restype = i32
        lib.cv_submit.argtypes = [vp, cv_buf, u64, ctypes.POINTER(u64)]
        lib.cv_submit.restype = i32
        lib.cv_poll.argtypes = [vp, u64, ctypes.c_int, ctypes.POINTER(vp)]
        lib.cv_poll.restype = i32
        lib.cv_server_get_stats.argtypes = [vp, ctypes.POINTER(cv_server_stats)]
        lib.cv_server_get_stats.restype = i32
        lib.cv_int_peak.argtypes = [ctypes.POINTER(cv_int_peak_info)]
        lib.cv_int_peak.restype = i32
        lib.cv_selftest_wait_timeout.argtypes = [u32, vp]
        lib.cv_selftest_wait_timeout.restype = i32
        lib.cv_probe_profile.argtypes = [vp, vp, u64, u64, ctypes.POINTER(cv_probe_stats), vp]
        lib.cv_probe_profile.restype = i32
        _lib = lib
        return lib


def strerror(code: int) -> str:
    return load().cv_strerror(code).decode()


def last_cuda_error() -> int:
    return int(load().cv_last_cuda_error())


def _check(rc: int, what: str) -> None:
    if rc != CV_OK:
        raise CVError(rc, what)


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _buf(x):
    """(pointer, n_bytes, keepalive) of a buffer-like object."""
    if isinstance(x, tuple):
        return int(x[0]), int(x[1]), None
    if hasattr(x, "data_ptr") and hasattr(x, "element_size"):  # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(x.data_ptr()), int(x.numel() * x.element_size()), x
    if isinstance(x, (bytes, bytearray, memoryview)):
        x = np.frombuffer(bytes(x), np.uint8)
    a = np.ascontiguousarray(x)
    return (int(a.ctypes.data) if a.size else 0), int(a.nbytes), a


def _bufs(xs):
    """A cv_buf array for a list of buffers. An (n, 2) uint64 array of (pointer, bytes) rows is
    passed as it is (it has cv_buf's layout), and a list made only of (pointer, bytes) tuples is
    converted in one step: with hundreds of thousands of master files the element-by-element
    path costs more than the build itself."""
    if isinstance(xs, np.ndarray):
        a = np.ascontiguousarray(xs, dtype=np.uint64)
        if a.ndim != 2 or a.shape[1] != 2:
            raise ValueError("a buffer descriptor array has shape (n, 2): pointer, bytes")
        return a.ctypes.data_as(ctypes.POINTER(cv_buf)), [a]
    if xs and all(type(x) is tuple for x in xs):
        a = np.array(xs, dtype=np.uint64)
        if a.ndim != 2 or a.shape[1] != 2:
            raise ValueError("buffer tuples are (pointer, bytes)")
        return a.ctypes.data_as(ctypes.POINTER(cv_buf)), [a]
    keep = []
    arr = (cv_buf * max(1, len(xs)))()
    for i, x in enumerate(xs):
        p, n, k = _buf(x)
        arr[i].data = p
        arr[i].n_bytes = n
        keep.append(k)
    return arr, keep


class Master:
    """A signature table of master files on the GPU (cv_master)."""

    def __init__(self, handle: int):
        self._h = handle

    @property
    def handle(self) -> int:
        return self._h

    def info(self) -> dict:
        inf = cv_master_info()
        _check(load().cv_master_get_info(self._h, ctypes.byref(inf)), "cv_master_get_info")
        return {k: getattr(inf, k) for k, _ in cv_master_info._fields_ if not k.startswith("reserved")}

    def close(self) -> None:
        if self._h:
            load().cv_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceMatches:
    """Matches of one image left in device memory; exposes __cuda_array_interface__ as an
    (n, 2) uint64 array: column 0 = disk_sector, column 1 = file_id | file_sector << 32."""

    def __init__(self, ptr: int, n: int, owner):
        self.ptr, self.n, self._owner = ptr, n, owner

    @property
    def __cuda_array_interface__(self):
        return {"shape": (self.n, 2), "typestr": "<u8", "data": (self.ptr or 0, False), "version": 3,
                "strides": None}


class Result:
    """Sorted matches of every scanned image (cv_result)."""

    def __init__(self, handle: int, n_images: int, on_device: bool):
        self._h = handle
        self.n_images = n_images
        self.on_device = on_device

    def _raw(self, i: int):
        p = ctypes.c_void_p()
        n = ctypes.c_uint64()
        _check(load().cv_matches(self._h, i, ctypes.byref(p), ctypes.byref(n)), "cv_matches")
        return p.value or 0, int(n.value)

    def matches(self, i: int = 0):
        """Image i's matches: a numpy structured array (host results) or DeviceMatches."""
        p, n = self._raw(i)
        if self.on_device:
            return DeviceMatches(p, n, self)
        if n == 0:
            return np.zeros(0, MATCH_DTYPE)
        buf = (ctypes.c_char * (n * 16)).from_address(p)
        return np.frombuffer(buf, MATCH_DTYPE, count=n).copy()

    def count(self, i: int = 0) -> int:
        return self._raw(i)[1]

    def stats(self) -> dict:
        st = cv_scan_stats()
        _check(load().cv_scan_get_stats(self._h, ctypes.byref(st)), "cv_scan_get_stats")
        return {k: getattr(st, k) for k, _ in cv_scan_stats._fields_}

    def close(self) -> None:
        if self._h:
            load().cv_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def master_build(files, max_load: float = 0.0, bloom_bits_per_key: int = CV_BLOOM_AUTO, stream=None,
                 signature: int = CV_SIG_MD5, position_mode: int = CV_POSITION_ANY,
                 layout: int = CV_LAYOUT_HASH, unit: int = CV_UNIT_SECTOR) -> Master:
    """cv_master_build: the signature table of a list of master files (one table over all sector
    positions, or with position_mode=CV_POSITION_CLUSTER the tables S_tau of Section 3.1), as a
    linear-probing hash table or (layout=CV_LAYOUT_SORTED) a sorted array searched by bisection.
    unit=CV_UNIT_FRAGMENT cuts the files into 64-byte fragments instead of 512-byte sectors, and
    scans then look up every 64-byte window at a 4-byte offset (Section 5). files: a list of
    buffers (arrays, tensors, (pointer, bytes) tuples) or an (n, 2) uint64 array of
    (pointer, bytes) rows."""
    files = files if isinstance(files, np.ndarray) else list(files)
    arr, keep = _bufs(files)
    o = cv_master_opts(ctypes.sizeof(cv_master_opts), max_load, bloom_bits_per_key, signature, _stream(stream),
                       position_mode, layout, unit, 0)
    h = ctypes.c_void_p()
    _check(load().cv_master_build(arr, len(files), ctypes.byref(o), ctypes.byref(h)), "cv_master_build")
    del keep
    return Master(h.value)


def master_save(master: Master, path) -> None:
    """cv_master_save: write the built table to a file."""
    _check(load().cv_master_save(master.handle, os.fsencode(path)), "cv_master_save")


def master_load(path, stream=None) -> Master:
    """cv_master_load: a table saved by master_save, checked and placed on the current device."""
    h = ctypes.c_void_p()
    _check(load().cv_master_load(os.fsencode(path), _stream(stream), ctypes.byref(h)), "cv_master_load")
    return Master(h.value)


def kernel_configs() -> list:
    """Names of the scan kernel configurations; index k is selected with kernel_config=k+1."""
    lib = load()
    return [lib.cv_kernel_config_name(k).decode() for k in range(lib.cv_kernel_config_count())]


def scan(master: Master, images, keep_on_device: bool = False, stream=None, chunk_bytes: int = 0,
         kernel_config: int = 0, base_offset: int = 0) -> Result:
    """cv_scan: every match of every image against the master table. base_offset: the disk sector
    where clusters start, for position-keyed tables."""
    images = list(images)
    arr, keep = _bufs(images)
    o = cv_scan_opts(ctypes.sizeof(cv_scan_opts), CV_KEEP_ON_DEVICE if keep_on_device else 0, _stream(stream),
                     chunk_bytes, kernel_config, 0, base_offset)
    h = ctypes.c_void_p()
    _check(load().cv_scan(master.handle, arr, len(images), ctypes.byref(o), ctypes.byref(h)), "cv_scan")
    del keep
    return Result(h.value, len(images), keep_on_device)


def sector_digests(in_ptr: int, n_sectors: int, out_ptr: int, trivial_ptr: int = 0, stream=None) -> None:
    """cv_sector_digests: MD5 of n_sectors device sectors into device memory (asynchronous)."""
    _check(load().cv_sector_digests(in_ptr, n_sectors, out_ptr, trivial_ptr or None, _stream(stream)),
           "cv_sector_digests")


def sector_signatures(in_ptr: int, n_sectors: int, signature: int, out_ptr: int, trivial_ptr: int = 0,
                      stream=None) -> None:
    """cv_sector_signatures: 16 bytes per device sector under any CV_SIG_* (asynchronous)."""
    _check(load().cv_sector_signatures(in_ptr, n_sectors, signature, out_ptr, trivial_ptr or None, _stream(stream)),
           "cv_sector_signatures")


def window_signatures(in_ptr: int, n_bytes: int, signature: int, out_ptr: int, stream=None) -> None:
    """cv_window_signatures: 16 bytes per 64-byte window at a 4-byte offset (asynchronous)."""
    _check(load().cv_window_signatures(in_ptr, n_bytes, signature, out_ptr, _stream(stream)),
           "cv_window_signatures")


def scan_noalloc(master: Master, image, out, out_capacity: int, stream=None, check: bool = True):
    """cv_scan_noalloc: scan one device image into a caller-owned device buffer of
    out_capacity matches, without any allocation. Returns (return code, match count); raises
    on any code other than CV_OK and CV_ERANGE when check is set."""
    ip, nb, _k1 = _buf(image)
    op, _, _k2 = _buf(out)
    n = ctypes.c_uint64()
    rc = load().cv_scan_noalloc(master.handle, ip, nb, op, out_capacity, ctypes.byref(n), _stream(stream))
    if check and rc not in (CV_OK, CV_ERANGE):
        raise CVError(rc, "cv_scan_noalloc")
    return rc, int(n.value)


class Batch:
    """Many device images scanned by one CUDA graph replay per run (cv_batch)."""

    def __init__(self, handle: int, n_images: int, keep):
        self._h = handle
        self.n_images = n_images
        self._keep = keep  # the images must outlive the batch

    def run(self, stream=None) -> None:
        _check(load().cv_batch_run(self._h, _stream(stream)), "cv_batch_run")

    def wait(self) -> int:
        n = ctypes.c_uint64()
        _check(load().cv_batch_wait(self._h, ctypes.byref(n)), "cv_batch_wait")
        return int(n.value)

    def matches(self, i: int) -> DeviceMatches:
        p = ctypes.c_void_p()
        n = ctypes.c_uint64()
        _check(load().cv_batch_matches(self._h, i, ctypes.byref(p), ctypes.byref(n)), "cv_batch_matches")
        return DeviceMatches(p.value or 0, int(n.value), self)

    def info(self) -> dict:
        inf = cv_batch_info()
        _check(load().cv_batch_get_info(self._h, ctypes.byref(inf)), "cv_batch_get_info")
        d = {k: getattr(inf, k) for k, _ in cv_batch_info._fields_ if k != "reserved"}
        d["config_name"] = d["config_name"].decode() if d["config_name"] else None
        return d

    def close(self) -> None:
        if self._h:
            load().cv_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_create(master: Master, images, autotune: bool = False, match_capacity: int = 0, kernel_config: int = 0,
                 bloom: int = CV_BATCH_BLOOM_AUTO, tune_cache: str | None = None, stream=None,
                 sorted_copy: bool = False) -> Batch:
    """cv_batch_create: a graph over device images (kept alive by the returned Batch)."""
    images = list(images)
    arr, keep = _bufs(images)
    o = cv_batch_opts(ctypes.sizeof(cv_batch_opts), 1 if autotune else 0, _stream(stream), match_capacity,
                      kernel_config, bloom, tune_cache.encode() if tune_cache else None, 1 if sorted_copy else 0, 0)
    h = ctypes.c_void_p()
    _check(load().cv_batch_create(master.handle, arr, len(images), ctypes.byref(o), ctypes.byref(h)),
           "cv_batch_create")
    return Batch(h.value, len(images), (images, keep))


def device_matches_to_numpy(dm: DeviceMatches) -> np.ndarray:
    """Copy device-resident matches to a host structured array (uses torch for the copy)."""
    import torch

    if dm.n == 0:
        return np.zeros(0, MATCH_DTYPE)
    t = torch.as_tensor(dm, device="cuda").cpu().numpy()
    out = np.zeros(t.shape[0], MATCH_DTYPE)
    out["disk_sector"] = t[:, 0]
    out["file_id"] = t[:, 1] & 0xFFFFFFFF
    out["file_sector"] = t[:, 1] >> 32
    return out


class Server:
    """A serving loop (cv_server): submit images as they arrive, poll their results."""

    def __init__(self, handle: int):
        self._h = handle
        self._keep = {}

    def submit(self, image, tag: int = 0) -> int:
        p, n, k = _buf(image)
        t = ctypes.c_uint64()
        _check(load().cv_submit(self._h, cv_buf(p, n), tag, ctypes.byref(t)), "cv_submit")
        self._keep[int(t.value)] = (image, k)
        return int(t.value)

    def poll(self, ticket: int, timeout_ms: int = -1):
        """The request's Result, or None if it is not done within timeout_ms."""
        h = ctypes.c_void_p()
        rc = load().cv_poll(self._h, ticket, timeout_ms, ctypes.byref(h))
        if rc == CV_EAGAIN:
            return None
        self._keep.pop(ticket, None)
        _check(rc, "cv_poll")
        return Result(h.value, 1, False)

    def stats(self) -> dict:
        st = cv_server_stats()
        _check(load().cv_server_get_stats(self._h, ctypes.byref(st)), "cv_server_get_stats")
        return {k: getattr(st, k) for k, _ in cv_server_stats._fields_}

    def close(self) -> None:
        if self._h:
            load().cv_free(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_create(master: Master, max_live: int = 0, hbm_budget_bytes: int = 0, work_unit_bytes: int = 0,
                  kernel_config: int = 0, copy_streams: int = 0, max_copy_bytes: int = 0) -> Server:
    """cv_server_create: a serving loop over one resident master table."""
    o = cv_server_opts(ctypes.sizeof(cv_server_opts), max_live, hbm_budget_bytes, work_unit_bytes, kernel_config,
                       copy_streams, max_copy_bytes)
    h = ctypes.c_void_p()
    _check(load().cv_server_create(master.handle, ctypes.byref(o), ctypes.byref(h)), "cv_server_create")
    return Server(h.value)


def int_peak() -> dict:
    """cv_int_peak: measured integer operation rates of this GPU."""
    inf = cv_int_peak_info()
    _check(load().cv_int_peak(ctypes.byref(inf)), "cv_int_peak")
    return {k: getattr(inf, k) for k, _ in cv_int_peak_info._fields_ if k != "reserved"}


def selftest_wait_timeout(timeout_us: int, stream=None) -> int:
    """cv_selftest_wait_timeout: return code of a bounded wait that runs out (CV_ETIMEOUT)."""
    return int(load().cv_selftest_wait_timeout(timeout_us, _stream(stream)))



def probe_profile(master: Master, image, base_offset: int = 0, stream=None) -> dict:
    """cv_probe_profile: exact table reads of the scan's lookups over one device image."""
    ip, nb, _k = _buf(image)
    st = cv_probe_stats()
    st.struct_size = ctypes.sizeof(cv_probe_stats)
    _check(load().cv_probe_profile(master.handle, ip, nb, base_offset, ctypes.byref(st), _stream(stream)),
           "cv_probe_profile")
    return {k: getattr(st, k) for k, _ in cv_probe_stats._fields_ if k != "struct_size"}
