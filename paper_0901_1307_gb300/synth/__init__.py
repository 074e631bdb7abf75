"""Seeded synthetic workloads: disk images and master files shaped like the paper's data.

Input generation only (no signature, table or matching arithmetic), shared by the tests, the
CPU oracle's inputs and the benchmark. Every byte is defined once in ``synth_def.h`` and produced
either on the host (``synth_host.c``, gcc) or on the device (``synth_cuda.cu``, nvcc); the two are
byte-identical, which the GPU tests check.

The paper scans disks whose 4 KiB clusters (8 sectors of 512 bytes, Section 2) may hold
fragments of known files; its experiments use random-data files (Section 4). A ``Plan`` places
a fraction of each master file's clusters at distinct cluster-aligned image positions, and
overwrites the first 1-4 sectors of some of them with fresh bytes (a newer file reusing the
cluster, Section 2). Every other sector is background: 70% random, 15% zero, 15% text.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

SECTOR = 512
CLUSTER = 8
TRIPLE_DTYPE = np.dtype([("disk_sector", "<u8"), ("file_id", "<u4"), ("file_sector", "<u4")])

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SRC = os.path.join(_HERE, "synth_host.c")
_CUDA_SRC = os.path.join(_HERE, "synth_cuda.cu")
_DEF = os.path.join(_HERE, "synth_def.h")
_HOST_LIB = os.path.join(_HERE, "libcvsynth.so")
_CUDA_LIB = os.path.join(_HERE, "libcvsynth_cuda.so")
_lock = threading.Lock()
_host = None
_cuda = None


def _stale(lib: str, srcs) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in srcs)


def build_host(force: bool = False) -> str:
    if force or _stale(_HOST_LIB, [_HOST_SRC, _DEF]):
        tmp = _HOST_LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-fopenmp", _HOST_SRC, "-o", tmp]
        try:
            subprocess.run(cmd, check=True, capture_output=True)
        except subprocess.CalledProcessError:
            cmd.remove("-fopenmp")
            subprocess.run(cmd, check=True, capture_output=True)
        os.replace(tmp, _HOST_LIB)
    return _HOST_LIB


def build_cuda(force: bool = False, nvcc: str = "nvcc") -> str:
    if force or _stale(_CUDA_LIB, [_CUDA_SRC, _DEF]):
        tmp = _CUDA_LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
               "-gencode", "arch=compute_103a,code=sm_103a", _CUDA_SRC, "-o", tmp]
        subprocess.run(cmd, check=True, capture_output=True)
        os.replace(tmp, _CUDA_LIB)
    return _CUDA_LIB


def _host_lib():
    global _host
    with _lock:
        if _host is None:
            lib = ctypes.CDLL(build_host())
            vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
            lib.synth_vocab.argtypes = [u64, vp]
            lib.synth_image.argtypes = [u64, u64, vp, vp, vp, u64, vp, vp, u64, u64, vp]
            lib.synth_master.argtypes = [u64, u32, u32, u32, vp]
            lib.synth_random.argtypes = [u64, u64, u64, u64, vp]
            lib.synth_hash.argtypes = [u64, u64, u64, u64]
            lib.synth_hash.restype = u64
            for f in (lib.synth_vocab, lib.synth_image, lib.synth_master, lib.synth_random):
                f.restype = None
            _host = lib
        return _host


def _cuda_lib():
    global _cuda
    with _lock:
        if _cuda is None:
            lib = ctypes.CDLL(build_cuda())
            vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
            lib.synth_image_cuda.argtypes = [u64, u64, vp, vp, vp, u64, vp, vp, u64, u64, vp, vp]
            lib.synth_image_cuda.restype = ctypes.c_int
            lib.synth_masters_cuda.argtypes = [u64, vp, u32, u64, vp, vp]
            lib.synth_masters_cuda.restype = ctypes.c_int
            _cuda = lib
        return _cuda


def sy_hash(seed: int, stream: int, a: int, b: int) -> int:
    return int(_host_lib().synth_hash(seed, stream, a, b))


def vocab(sigma: int) -> np.ndarray:
    out = np.zeros(2000 * 16, np.uint8)
    _host_lib().synth_vocab(sigma, out.ctypes.data)
    return out


def random_sectors(seed: int, n: int, first: int = 0, stream: int = 99) -> np.ndarray:
    """n fresh random sectors (uint8, n*512) that no master or image stream produces."""
    out = np.zeros(n * SECTOR, np.uint8)
    if n:
        _host_lib().synth_random(seed, stream, first, n, out.ctypes.data)
    return out


@dataclasses.dataclass
class Plan:
    """One synthetic image and its master set."""

    image_seed: int
    master_seed: int
    n_sectors: int
    file_nsect: np.ndarray      # uint32 [n_files]: whole sectors per master file
    plant_file: np.ndarray      # int32 [n_clusters]: planted file id or -1
    plant_fcluster: np.ndarray  # uint32 [n_clusters]
    plant_over: np.ndarray      # uint8 [n_clusters]: leading sectors overwritten

    @property
    def n_files(self) -> int:
        return int(self.file_nsect.size)

    @property
    def n_master_sectors(self) -> int:
        return int(self.file_nsect.sum(dtype=np.uint64))

    @property
    def n_bytes(self) -> int:
        return self.n_sectors * SECTOR

    def file_base(self) -> np.ndarray:
        base = np.zeros(self.n_files + 1, np.uint64)
        np.cumsum(self.file_nsect, dtype=np.uint64, out=base[1:])
        return base

    # ------------------------------------------------------------------ host generation
    def _args(self):
        self._vocab = vocab(self.image_seed)
        return (self.image_seed, self.master_seed, self.plant_file.ctypes.data, self.plant_fcluster.ctypes.data,
                self.plant_over.ctypes.data, self.plant_file.size, self.file_nsect.ctypes.data,
                self._vocab.ctypes.data)

    def image_host(self, first: int = 0, n: int | None = None) -> np.ndarray:
        """Image sectors [first, first+n) as uint8 (n*512)."""
        if n is None:
            n = self.n_sectors - first
        out = np.zeros(n * SECTOR, np.uint8)
        if n:
            _host_lib().synth_image(*self._args(), first, n, out.ctypes.data)
        return out

    def image_host_into(self, out_ptr: int, first: int, n: int) -> None:
        """Write image sectors [first, first+n) to host memory at out_ptr (n*512 bytes), e.g. a
        slot of a pinned pool; the host generator runs on all cores (OpenMP)."""
        if n:
            _host_lib().synth_image(*self._args(), first, n, out_ptr)

    def master_host(self, f: int, s0: int = 0, n: int | None = None) -> np.ndarray:
        if n is None:
            n = int(self.file_nsect[f]) - s0
        out = np.zeros(n * SECTOR, np.uint8)
        if n:
            _host_lib().synth_master(self.master_seed, f, s0, n, out.ctypes.data)
        return out

    def masters_host(self) -> list:
        """Every master file as a uint8 array (whole sectors)."""
        return [self.master_host(f) for f in range(self.n_files)]

    # ---------------------------------------------------------------- device generation
    def image_device(self, out_ptr: int, first: int = 0, n: int | None = None, stream: int = 0,
                     dev_plan=None) -> None:
        """Write image sectors [first, first+n) to device memory at out_ptr (8-byte aligned).

        dev_plan is the tuple returned by ``device_plan`` (device copies of the plan arrays,
        kept alive by the caller)."""
        if n is None:
            n = self.n_sectors - first
        pf, pc, po, fn, vc = dev_plan
        rc = _cuda_lib().synth_image_cuda(self.image_seed, self.master_seed, pf, pc, po, self.plant_file.size,
                                          fn, vc, first, n, out_ptr, stream)
        if rc != 0:
            raise RuntimeError(f"synth_image_cuda failed: cuda error {rc}")

    def masters_device(self, out_ptr: int, file_base_ptr: int, stream: int = 0) -> None:
        """All master files concatenated (file order, whole sectors) into device memory."""
        rc = _cuda_lib().synth_masters_cuda(self.master_seed, file_base_ptr, self.n_files,
                                            self.n_master_sectors, out_ptr, stream)
        if rc != 0:
            raise RuntimeError(f"synth_masters_cuda failed: cuda error {rc}")

    # --------------------------------------------------------------------- plant log
    def planted(self) -> np.ndarray:
        """Image cluster indices that carry a planted master cluster."""
        return np.nonzero(self.plant_file >= 0)[0]

    def expected_intact(self) -> np.ndarray:
        """Every planted master sector that survived the overwrites, as sorted triples.

        This is a subset of the match result (exactly the result when master sectors are
        random and unique, as in every configuration here)."""
        q = self.planted()
        if q.size == 0:
            return np.zeros(0, TRIPLE_DTYPE)
        f = self.plant_file[q].astype(np.int64)
        c = self.plant_fcluster[q].astype(np.int64)
        ov = self.plant_over[q].astype(np.int64)
        k = np.arange(CLUSTER, dtype=np.int64)
        s = c[:, None] * CLUSTER + k[None, :]
        i = q.astype(np.int64)[:, None] * CLUSTER + k[None, :]
        keep = (k[None, :] >= ov[:, None]) & (s < self.file_nsect[f][:, None].astype(np.int64)) & (i < self.n_sectors)
        out = np.zeros(int(keep.sum()), TRIPLE_DTYPE)
        out["disk_sector"] = i[keep]
        out["file_id"] = np.broadcast_to(f[:, None], s.shape)[keep]
        out["file_sector"] = s[keep]
        out.sort(order=["disk_sector", "file_id", "file_sector"])
        return out


def make_plan(image_seed: int, n_sectors: int, file_nsect, plant_frac: float, overwrite_frac: float = 0.10,
              master_seed: int | None = None, plan_seed: int | None = None) -> Plan:
    """Place round(plant_frac * clusters) clusters of every master file at distinct, uniformly
    drawn cluster-aligned image positions; overwrite the first 1-4 sectors of
    round(overwrite_frac * planted) of them."""
    file_nsect = np.asarray(file_nsect, dtype=np.uint32)
    master_seed = image_seed + 0x5EED if master_seed is None else master_seed
    rng = np.random.default_rng([image_seed, 0xC1A5] if plan_seed is None else plan_seed)
    n_clusters = (n_sectors + CLUSTER - 1) // CLUSTER
    files, fcl = [], []
    for f, ns in enumerate(file_nsect.tolist()):
        nc = (ns + CLUSTER - 1) // CLUSTER
        k = int(round(plant_frac * nc))
        if k:
            chosen = np.sort(rng.choice(nc, size=k, replace=False))
            files.append(np.full(k, f, np.int32))
            fcl.append(chosen.astype(np.uint32))
    plant_file = np.full(n_clusters, -1, np.int32)
    plant_fcluster = np.zeros(n_clusters, np.uint32)
    plant_over = np.zeros(n_clusters, np.uint8)
    if files:
        pf = np.concatenate(files)
        pc = np.concatenate(fcl)
        P = pf.size
        if P > n_clusters:
            raise ValueError(f"{P} planted clusters do not fit in {n_clusters} image clusters")
        slots = rng.choice(n_clusters, size=P, replace=False)
        plant_file[slots] = pf
        plant_fcluster[slots] = pc
        n_over = int(round(overwrite_frac * P))
        if n_over:
            which = rng.choice(P, size=n_over, replace=False)
            plant_over[slots[which]] = rng.integers(1, 5, size=n_over).astype(np.uint8)
    return Plan(image_seed, master_seed, n_sectors, file_nsect, plant_file, plant_fcluster, plant_over)


def make_plan_density(image_seed: int, n_sectors: int, file_nsect, density: float, master_seed: int,
                      overwrite_frac: float = 0.10) -> Plan:
    """Plant round(density * image clusters) distinct image clusters, each with a master cluster
    drawn uniformly over every cluster of every master file (repeats allowed), and overwrite the
    first 1-4 sectors of round(overwrite_frac * planted) of them."""
    file_nsect = np.asarray(file_nsect, dtype=np.uint32)
    rng = np.random.default_rng([image_seed, 0xD3])
    n_clusters = (n_sectors + CLUSTER - 1) // CLUSTER
    plant_file = np.full(n_clusters, -1, np.int32)
    plant_fcluster = np.zeros(n_clusters, np.uint32)
    plant_over = np.zeros(n_clusters, np.uint8)
    P = int(round(density * n_clusters))
    if P and file_nsect.size:
        slots = rng.choice(n_clusters, size=P, replace=False)
        ncl = (file_nsect.astype(np.int64) + CLUSTER - 1) // CLUSTER
        cum = np.cumsum(ncl)
        g = rng.integers(0, int(cum[-1]), size=P)
        f = np.searchsorted(cum, g, side="right")
        c = g - (cum[f] - ncl[f])
        plant_file[slots] = f.astype(np.int32)
        plant_fcluster[slots] = c.astype(np.uint32)
        n_over = int(round(overwrite_frac * P))
        if n_over:
            which = rng.choice(P, size=n_over, replace=False)
            plant_over[slots[which]] = rng.integers(1, 5, size=n_over).astype(np.uint8)
    return Plan(image_seed, master_seed, n_sectors, file_nsect, plant_file, plant_fcluster, plant_over)


def master_set(name: str):
    """(file_nsect, master_seed) of a named master set.

    m8m: 40,000 files with log-uniform 8 KiB-1 MiB sizes scaled to 8,388,608 sectors, seed 4
         (the shared table of the batched and served workloads)."""
    if name == "m8m":
        rng = np.random.default_rng(4)
        raw = log_uniform_sizes(rng, 40000, 8 << 10, 1 << 20) / SECTOR
        return scale_to_total(raw, 8388608, 16), 4 + 0x5EED
    raise KeyError(name)


def sweep_master_set(m_sectors: int):
    """(file_nsect, master_seed) of the table-scaling sweep: the scale workload's file-size
    distribution (log-uniform 8 KiB-1 MiB, about 210 sectors per file) scaled to m_sectors whole
    sectors, seed 3."""
    n_files = max(1, int(round(m_sectors / 210)))
    rng = np.random.default_rng([3, m_sectors])
    raw = log_uniform_sizes(rng, n_files, 8 << 10, 1 << 20) / SECTOR
    return scale_to_total(raw, m_sectors, min(16, m_sectors // n_files)), 3 + 0x5EED + m_sectors


def batch_sizes(seed: int, n: int, lo_bytes: int, hi_bytes: int, total_bytes: int) -> np.ndarray:
    """Image sizes in sectors: log-uniform lo..hi, scaled to total_bytes, each at least lo_bytes
    and a whole number of 4 KiB clusters."""
    rng = np.random.default_rng(seed)
    raw = log_uniform_sizes(rng, n, lo_bytes, hi_bytes)
    raw = raw * (total_bytes / raw.sum())
    clusters = np.maximum(np.round(raw / (CLUSTER * SECTOR)), lo_bytes // (CLUSTER * SECTOR)).astype(np.int64)
    diff = total_bytes // (CLUSTER * SECTOR) - int(clusters.sum())
    order = np.argsort(-clusters)
    i = 0
    while diff != 0:
        j = order[i % n]
        step = 1 if diff > 0 else -1
        if clusters[j] + step >= lo_bytes // (CLUSTER * SECTOR):
            clusters[j] += step
            diff -= step
        i += 1
    return clusters * CLUSTER


def log_uniform_sizes(rng, n: int, lo_bytes: int, hi_bytes: int) -> np.ndarray:
    return np.exp(rng.uniform(np.log(lo_bytes), np.log(hi_bytes), size=n))


def scale_to_total(sizes_sectors: np.ndarray, total: int, min_sectors: int) -> np.ndarray:
    """Scale sizes by a common factor so they sum exactly to ``total`` whole sectors."""
    s = np.maximum(np.round(sizes_sectors * (total / sizes_sectors.sum())), min_sectors).astype(np.int64)
    diff = total - int(s.sum())
    order = np.argsort(-s)
    i = 0
    while diff != 0:
        j = order[i % s.size]
        step = 1 if diff > 0 else -1
        if s[j] + step >= min_sectors:
            s[j] += step
            diff -= step
        i += 1
    return s.astype(np.uint32)


def config_plan(name: str) -> Plan:
    """The named workloads.

    tiny  : 64 MiB image (131,072 sectors), seed 0; 150 master files of uniform 16-256 KiB
            (32-512 sectors); 40% of each file's clusters planted, 10% of those partly overwritten.
    scale : 32 GiB image (67,108,864 sectors), seed 1; 20,000 master files with log-uniform
            8 KiB-1 MiB sizes scaled to 4,194,304 sectors in total (minimum 16); 25% planted.
    mid   : 4 GiB image (8,388,608 sectors), seed 6; 1,250 such files scaled to 262,144 sectors.
    """
    if name == "tiny":
        rng = np.random.default_rng(0)
        nsect = rng.integers(32, 513, size=150)
        return make_plan(0, 131072, nsect, 0.40)
    if name == "scale":
        rng = np.random.default_rng(1)
        raw = log_uniform_sizes(rng, 20000, 8 << 10, 1 << 20) / SECTOR
        nsect = scale_to_total(raw, 4194304, 16)
        return make_plan(1, 67108864, nsect, 0.25)
    if name == "mid":
        # a 4 GiB image against 262,144 master sectors: the scale workload's mix at 1/8 of the
        # image and 1/16 of the masters, for profiling runs
        rng = np.random.default_rng(6)
        raw = log_uniform_sizes(rng, 1250, 8 << 10, 1 << 20) / SECTOR
        nsect = scale_to_total(raw, 262144, 16)
        return make_plan(6, 8388608, nsect, 0.25)
    if name.startswith("small:"):
        # small:<sectors>:<files>:<seed> -- a scaled-down image for fast tests
        _, ns, nf, seed = name.split(":")
        rng = np.random.default_rng(int(seed))
        nsect = rng.integers(16, 129, size=int(nf))
        return make_plan(int(seed), int(ns), nsect, 0.40)
    raise KeyError(name)


# ----------------------------------------------------------------------------------------------
# Fragment workloads (Section 5: every 64-byte fragment at a 32-bit boundary, to find small
# images and logos embedded in documents).

FRAG = 64
FRAG_STRIDE = 4
_LOGO_STREAM = 101
_HEADER_STREAM = 102


@dataclasses.dataclass
class FragPlan:
    """Small master files ("logos") embedded at 4-byte-aligned offsets of a background image.

    Logos are random bytes; some start with a header shared by several logos (so one fragment
    belongs to several files) and some hold a zero-filled run at a fragment boundary (fragments
    the exclusion rule drops). Planted copies do not overlap one another."""

    background: Plan           # the image's background: the three sector classes, nothing planted
    n_bytes: int               # image length (need not be a multiple of 512 or 4)
    logo_seed: int
    logo_bytes: np.ndarray     # int64 [n_logos]
    header_len: np.ndarray     # int64 [n_logos]: bytes of the shared header at the logo's start
    zero_at: np.ndarray        # int64 [n_logos]: fragment index of a zero run (-1: none)
    zero_len: np.ndarray       # int64 [n_logos]: its length in bytes
    plant_logo: np.ndarray     # int64 [n_plants]
    plant_off: np.ndarray      # int64 [n_plants]: byte offsets, multiples of 4

    @property
    def n_logos(self) -> int:
        return int(self.logo_bytes.size)

    def _header(self) -> np.ndarray:
        n = int(self.header_len.max()) if self.n_logos else 0
        return random_sectors(self.logo_seed, (n + SECTOR - 1) // SECTOR, 0, _HEADER_STREAM)[:n]

    def logo(self, f: int, header: np.ndarray | None = None) -> np.ndarray:
        nb = int(self.logo_bytes[f])
        first = int(np.sum(((self.logo_bytes[:f] + SECTOR - 1) // SECTOR)))
        out = random_sectors(self.logo_seed, (nb + SECTOR - 1) // SECTOR, first, _LOGO_STREAM)[:nb].copy()
        h = int(self.header_len[f])
        if h:
            out[:h] = (self._header() if header is None else header)[:h]
        if self.zero_at[f] >= 0:
            z = int(self.zero_at[f]) * FRAG
            out[z:z + int(self.zero_len[f])] = 0
        return out

    def logos(self) -> list:
        header = self._header()
        return [self.logo(f, header) for f in range(self.n_logos)]

    def image_host(self) -> np.ndarray:
        img = self.background.image_host()[: self.n_bytes].copy()
        logos = self.logos()
        for f, o in zip(self.plant_logo.tolist(), self.plant_off.tolist()):
            img[o:o + logos[f].size] = logos[f]
        return img

    def image_device(self, torch, out) -> None:
        """Write the image into the uint8 device tensor out (at least n_bytes long)."""
        bg = self.background
        pf, pc, po = (torch.from_numpy(a).cuda() for a in (bg.plant_file, bg.plant_fcluster.view(np.int32),
                                                            bg.plant_over))
        fn = torch.zeros(1, dtype=torch.int32).cuda()
        vc = torch.from_numpy(vocab(bg.image_seed)).cuda()
        bg.image_device(out.data_ptr(), 0, self.n_bytes // SECTOR,
                        dev_plan=(pf.data_ptr(), pc.data_ptr(), po.data_ptr(), fn.data_ptr(), vc.data_ptr()))
        tail = self.n_bytes % SECTOR
        if tail:
            out[self.n_bytes - tail:self.n_bytes].copy_(torch.from_numpy(bg.image_host(self.n_bytes // SECTOR, 1)[:tail]))
        logos = self.logos()
        sizes = np.array([x.size for x in logos], np.int64)
        base = np.zeros(self.n_logos + 1, np.int64)
        np.cumsum(sizes, out=base[1:])
        flat = torch.from_numpy(np.concatenate(logos) if logos else np.zeros(0, np.uint8)).cuda()
        for f, o in zip(self.plant_logo.tolist(), self.plant_off.tolist()):
            out[o:o + int(sizes[f])].copy_(flat[int(base[f]):int(base[f + 1])])
        torch.cuda.synchronize()

    def expected_planted(self) -> np.ndarray:
        """Triples (window, logo, fragment) of every planted logo's whole, non-zero-run fragments:
        a subset of the result (logos are random, so the result adds only the other files that
        share a header fragment)."""
        rows = []
        for f, o in zip(self.plant_logo.tolist(), self.plant_off.tolist()):
            n_fr = int(self.logo_bytes[f]) // FRAG
            j = np.arange(n_fr, dtype=np.int64)
            if self.zero_at[f] >= 0:
                z0, z1 = int(self.zero_at[f]) * FRAG, int(self.zero_at[f]) * FRAG + int(self.zero_len[f])
                j = j[~((j * FRAG >= z0) & ((j + 1) * FRAG <= z1))]
            t = np.zeros(j.size, TRIPLE_DTYPE)
            t["disk_sector"] = o // FRAG_STRIDE + j * (FRAG // FRAG_STRIDE)
            t["file_id"] = f
            t["file_sector"] = j
            rows.append(t)
        out = np.concatenate(rows) if rows else np.zeros(0, TRIPLE_DTYPE)
        out.sort(order=["disk_sector", "file_id", "file_sector"])
        return out


def make_frag_plan(seed: int, n_bytes: int, n_logos: int, lo_bytes: int = 1024, hi_bytes: int = 16384,
                   header_frac: float = 0.1, header_bytes: int = 128, zero_frac: float = 0.2,
                   plant_frac: float = 0.5, max_copies: int = 3) -> FragPlan:
    """n_logos logos of log-uniform lo..hi bytes; header_frac of them start with a shared
    header_bytes header, zero_frac hold a zero run of 64-192 bytes at a fragment boundary;
    plant_frac of them are planted 1..max_copies times at non-overlapping 4-byte-aligned
    offsets of an n_bytes image whose background is the usual sector mix."""
    rng = np.random.default_rng([seed, 0xF4A6])
    sizes = np.round(log_uniform_sizes(rng, n_logos, lo_bytes, hi_bytes)).astype(np.int64)
    header_len = np.where(rng.random(n_logos) < header_frac, min(header_bytes, lo_bytes), 0).astype(np.int64)
    zero_at = np.full(n_logos, -1, np.int64)
    zero_len = np.zeros(n_logos, np.int64)
    for f in np.nonzero(rng.random(n_logos) < zero_frac)[0].tolist():
        n_fr = int(sizes[f]) // FRAG
        if n_fr >= 4:
            zero_at[f] = int(rng.integers(2, n_fr - 1))
            zero_len[f] = FRAG * int(rng.integers(1, 4))
    planted = np.nonzero(rng.random(n_logos) < plant_frac)[0]
    plants = np.repeat(planted, rng.integers(1, max_copies + 1, size=planted.size))
    rng.shuffle(plants)
    P = plants.size
    offs = np.zeros(P, np.int64)
    if P:
        region = (n_bytes // P) // FRAG_STRIDE * FRAG_STRIDE
        if region < int(sizes[plants].max()):
            raise ValueError("image too small for the planted logos")
        room = (region - sizes[plants]) // FRAG_STRIDE
        offs = np.arange(P, dtype=np.int64) * region + FRAG_STRIDE * rng.integers(0, room + 1)
    n_sectors = (n_bytes + SECTOR - 1) // SECTOR
    background = make_plan(seed, n_sectors, np.zeros(0, np.uint32), 0.0)
    return FragPlan(background, n_bytes, seed + 0x10CC, sizes, header_len, zero_at, zero_len,
                    plants.astype(np.int64), offs)


def frag_config(name: str) -> FragPlan:
    """The named fragment workloads.

    frag  : 4 GiB image, seed 11; 2,000 logos of log-uniform 1-16 KiB, half planted 1-3 times.
    frag_small:<bytes>:<logos>:<seed> -- scaled down for tests."""
    if name == "frag":
        return make_frag_plan(11, 4 << 30, 2000)
    if name.startswith("frag_small:"):
        _, nb, nl, seed = name.split(":")
        return make_frag_plan(int(seed), int(nb), int(nl))
    raise KeyError(name)
