"""Benchmark: disk-image GB/s scanned on one GB300 through the C ABI.

Workload ("scale"): a 32 GiB synthetic disk image (67,108,864 sectors of 512 bytes: 70% random,
15% zero, 15% text sectors) against 20,000 master files totalling 4,194,304 sectors (log-uniform
8 KiB-1 MiB, scaled), 25% of whose 4 KiB clusters are planted in the image, 10% of those partly
overwritten. The image and masters are generated on the device (seeded, synth module) before
timing; the image is larger than L2, so no flush is needed between steps.

A step is one cv_scan call on the device-resident image: hashing + Bloom + probe + compaction,
the sorted match list left in device memory. value = image bytes / device time (CUDA events on
the scan stream). e2e = the same call on the image in pinned host memory, host-to-device copies
and the device-to-host copy of the matches inside the timed region.

--impl reference times the CPU oracle (the method written plainly, OpenMP over host cores) on
bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SECTOR = 512
MD5_OPS_PER_SECTOR = 2852  # 8 data blocks x 64 ops x 5 + padding block 64 x 4 + 9 x 4 feed-forward
SM_COUNT = 152
INT_LANES_PER_SM_CLK = 128  # 4 schedulers x 32 lanes, integer work split over the ALU and FMA pipes


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """The largest value over all ranks (the step time of the slowest rank); no collective on
    the data path, only this reduction of one number."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def image_on_device(torch, synth, plan):
    """The plan's image generated in device memory."""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    keep = [dev(plan.plant_file.view(np.uint8)), dev(plan.plant_fcluster.view(np.uint8)), dev(plan.plant_over),
            dev(plan.file_nsect.view(np.uint8)), dev(synth.vocab(plan.image_seed))]
    image = torch.empty(plan.n_bytes, dtype=torch.uint8, device="cuda")
    plan.image_device(image.data_ptr(), dev_plan=tuple(k.data_ptr() for k in keep))
    torch.cuda.synchronize()
    return image


def setup_workload(torch, cv, synth, name: str, seed_offset: int, signature: int = 0):
    plan = synth.config_plan(name)
    if seed_offset:
        plan.image_seed += seed_offset
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    image = image_on_device(torch, synth, plan)
    keep = []
    base = plan.file_base()
    base_d = dev(base.view(np.uint8))
    masters = torch.empty(plan.n_master_sectors * SECTOR, dtype=torch.uint8, device="cuda")
    plan.masters_device(masters.data_ptr(), base_d.data_ptr())
    torch.cuda.synchronize()
    files = file_descriptors(masters.data_ptr(), base, plan.file_nsect)
    t0 = time.perf_counter()
    master = cv.master_build(files, signature=signature)
    build_s = time.perf_counter() - t0
    del masters, keep
    torch.cuda.synchronize()
    return plan, image, master, build_s


def cpu_baseline(plan, pieces: int):
    """The oracle's lookup timed on `pieces` 1 GiB windows of the image at seeded offsets."""
    import oracle

    files = plan.masters_host()
    db = oracle.OracleDB(files)
    n = min(1 << 21, plan.n_sectors)
    rng = np.random.default_rng(12345)
    starts = sorted(rng.integers(0, plan.n_sectors - n + 1, size=pieces).tolist())
    secs, found = 0.0, 0
    for s in starts:
        img = plan.image_host(int(s), n)
        t0 = time.perf_counter()
        found += db.lookup(img, int(s)).size
        secs += time.perf_counter() - t0
    # the same lookup on one host core, over the first window only
    cores = oracle.threads()
    img = plan.image_host(int(starts[0]), n)
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        db.lookup(img, int(starts[0]))
        one = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    db.close()
    return {"value": pieces * n * SECTOR / secs / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{pieces} windows of {n} sectors ({n * SECTOR / 2**30:.0f} GiB each) at seeded offsets of "
                      f"the image; lookup only, signature database of {plan.n_master_sectors} master sectors "
                      f"built untimed", "matches_in_sample": found, "seconds": secs,
            "single_core_GBps": n * SECTOR / one / 1e9}


def run_reference(args):
    rank, world, local = rank_env()
    if rank != 0:
        return 0
    from paper_0901_1307_gb300 import synth
    import oracle

    plan = synth.config_plan(args.config)
    files = plan.masters_host()
    db = oracle.OracleDB(files)
    n = args.ref_sample_sectors
    rng = np.random.default_rng(0)
    starts = rng.integers(0, plan.n_sectors - n, size=args.warmup + args.steps)
    times = []
    for k, s in enumerate(starts):
        img = plan.image_host(int(s), n)
        t0 = time.perf_counter()
        db.lookup(img, int(s))
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    v = args.steps * n * SECTOR / tot / 1e9
    line = {"metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{args.config}: 32 GiB image, 4,194,304 master sectors, oracle sample of "
                                   f"{n} sectors per step", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{n} random-offset sectors per step"},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    db.close()
    print(json.dumps(line), flush=True)
    return 0


def device_plan(torch, synth, plan):
    """Device copies of a plan's arrays (the generator reads them); keep the list alive."""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    keep = [dev(plan.plant_file.view(np.uint8)), dev(plan.plant_fcluster.view(np.uint8)), dev(plan.plant_over),
            dev(plan.file_nsect.view(np.uint8)), dev(synth.vocab(plan.image_seed))]
    return tuple(k.data_ptr() for k in keep), keep


def file_descriptors(ptr, base, file_nsect):
    """(pointer, bytes) rows of files laid out from ptr at sector offsets base (a cv_buf array)."""
    n = file_nsect.size
    return np.stack([ptr + base[:n].astype(np.uint64) * SECTOR, file_nsect.astype(np.uint64) * SECTOR], axis=1)


def build_master_set(torch, cv, synth, name):
    """The named master set generated on the device and built into a table."""
    file_nsect, mseed = synth.master_set(name)
    mplan = synth.Plan(0, mseed, 0, file_nsect, np.zeros(0, np.int32), np.zeros(0, np.uint32), np.zeros(0, np.uint8))
    base = mplan.file_base()
    base_d = torch.from_numpy(base.view(np.uint8).copy()).cuda()
    masters = torch.empty(mplan.n_master_sectors * SECTOR, dtype=torch.uint8, device="cuda")
    mplan.masters_device(masters.data_ptr(), base_d.data_ptr())
    torch.cuda.synchronize()
    files = file_descriptors(masters.data_ptr(), base, file_nsect)
    t0 = time.perf_counter()
    m = cv.master_build(files)
    build_s = time.perf_counter() - t0
    del masters
    torch.cuda.synchronize()
    return m, file_nsect, mseed, build_s


def expected_window(expect: np.ndarray, a: int, n: int) -> np.ndarray:
    """The triples of disk sectors [a, a + n) renumbered from 0."""
    lo = np.searchsorted(expect["disk_sector"], a, side="left")
    hi = np.searchsorted(expect["disk_sector"], a + n, side="left")
    out = expect[lo:hi].copy()
    out["disk_sector"] -= a
    return out


def run_signatures(torch, cv, synth, plan, image, stream, steps):
    """The same device-resident scan with the paper's other signatures: MD5 without padding,
    djb2-64 and CRC64 (64-bit ones confirmed byte for byte on the device), each with its default
    kernel configuration and each result checked against the plant log."""
    masters, files = device_masters(torch, plan)
    out = {}
    want = plan.expected_intact()
    names = cv.kernel_configs()
    for sig, name in ((0, "md5"), (1, "md5_nopad"), (2, "djb2_64"), (3, "crc64")):
        m = cv.master_build(files, signature=sig)
        wall, kms, matches = time_scans(torch, cv, m, image, stream, steps)
        r = cv.scan(m, [image], stream=stream)
        exact = bool(np.array_equal(r.matches(0), want))
        st = r.stats()
        r.close()
        out[name] = {"GBps": plan.n_bytes / wall / 1e9, "kernel_GBps": plan.n_bytes / (kms * 1e-3) / 1e9,
                     "matches": matches, "bit_exact_vs_plant_log": exact, "kernel_config": names[st["kernel_config"]],
                     "confirm_rejected": st["confirm_rejected"]}
        m.close()
    # the paper's position-keyed tables S_tau on the same image (clusters from sector 0)
    m = cv.master_build(files, position_mode=cv.CV_POSITION_CLUSTER)
    wall, kms, matches = time_scans(torch, cv, m, image, stream, steps)
    out["md5_position_tau"] = {"GBps": plan.n_bytes / wall / 1e9, "kernel_GBps": plan.n_bytes / (kms * 1e-3) / 1e9,
                               "matches": matches}
    m.close()
    del masters
    torch.cuda.synchronize()
    return out


def device_masters(torch, plan):
    """The plan's master files generated on the device: (arena tensor, [(ptr, bytes)] per file)."""
    base = plan.file_base()
    base_d = torch.from_numpy(base.view(np.uint8).copy()).cuda()
    masters = torch.empty(plan.n_master_sectors * SECTOR, dtype=torch.uint8, device="cuda")
    plan.masters_device(masters.data_ptr(), base_d.data_ptr())
    torch.cuda.synchronize()
    files = file_descriptors(masters.data_ptr(), base, plan.file_nsect)
    return masters, files


def time_scans(torch, cv, m, image, stream, steps):
    """Mean wall and kernel time of `steps` device-resident scans (after 3 untimed ones)."""
    for _ in range(3):
        cv.scan(m, [image], keep_on_device=True, stream=stream).close()
    kms, matches = [], 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        r = cv.scan(m, [image], keep_on_device=True, stream=stream)
        st = r.stats()
        kms.append(st["kernel_ms"])
        matches = st["matches"]
        r.close()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / steps, statistics.mean(kms), matches


def run_tables(torch, cv, synth, plan, image, stream, steps):
    """Throughput against table occupancy (as the paper plots it for CRC64 and djb2), for the
    linear-probing hash table and the sorted table searched by bisection, with and without the
    Bloom filter. Occupancy is set by the number of master sectors in a 2^22-slot table: a
    prefix of the master files holding about occ x 2^22 sectors."""
    masters, files = device_masters(torch, plan)
    cum = np.cumsum(plan.file_nsect.astype(np.int64))
    slots = 1 << 22
    out = {}
    for occ in (0.25, 0.5, 0.75, 0.9):
        k = max(int(np.searchsorted(cum, occ * (slots - 1) * 0.999, side="right")), 1)
        sub = files[:k]
        # the load cap that sizes the table at exactly 2^22 slots for these sectors
        max_load = min(0.9, float(cum[k - 1]) / (slots * 0.9999))
        # MD5 with both layouts, Bloom on and off; the paper's measured signatures (djb2-64, CRC64)
        # as it ran them, without a Bloom filter, with both layouts
        variants = [(0, layout, bloom) for layout in (0, 1) for bloom in (0, 16)]
        variants += [(sig, layout, 0) for sig in (2, 3) for layout in (0, 1)]
        for sig, layout, bloom in variants:
            m = cv.master_build(sub, max_load=max_load, layout=layout, bloom_bits_per_key=bloom, signature=sig)
            info = m.info()
            wall, kms, matches = time_scans(torch, cv, m, image, stream, steps)
            # exact table reads of the lookups, on the image's first 2 GiB (4,194,304 sectors)
            prof = image[: 1 << 31]
            pr = cv.probe_profile(m, prof, stream=stream)
            ns = prof.numel() // SECTOR
            sname = {0: "", 2: "djb2_", 3: "crc64_"}[sig]
            lname = "sorted" if layout else "hash"
            out[f"occ{occ}_{sname}{lname}_{'bloom' if bloom else 'nobloom'}"] = {
                "occupancy": info["n_unique"] / max(info["n_slots"], 1), "n_slots": info["n_slots"],
                "master_sectors": int(cum[k - 1]), "signature": sig,
                "max_probe_or_steps": info["max_probe"], "GBps": plan.n_bytes / wall / 1e9,
                "kernel_GBps": plan.n_bytes / (kms * 1e-3) / 1e9, "matches": matches,
                "bloom_pass_per_sector": pr["bloom_passed"] / ns, "slot_reads_per_sector": pr["slot_reads"] / ns,
                "key_reads_per_sector": pr["key_reads"] / ns,
                "slot_reads_per_lookup": pr["slot_reads"] / max(pr["bloom_passed"], 1)}
            m.close()
    del masters
    torch.cuda.synchronize()
    return out


# DRAM bytes (read + write) per launch of the default scan kernel, from one ncu capture of the
# current kernel: 4.3773 GB on the 4 GiB mid workload (8,388,608 sectors; the mean of four
# launches), scaled by sectors.
SCAN_TRAFFIC_BYTES = {"mid": 4.3773e9, "scale": 8 * 4.3773e9}


def run_build(torch, cv, synth, M, reps=3):
    """Table builds (cv_master_build, MD5, Bloom filter) of the sweep's master set of M sectors,
    device-resident, as many files as that set has; the first build is a warm-up."""
    file_nsect, mseed = synth.sweep_master_set(M)
    mplan = synth.Plan(0, mseed, 0, file_nsect, np.zeros(0, np.int32), np.zeros(0, np.uint32), np.zeros(0, np.uint8))
    base = mplan.file_base()
    base_d = torch.from_numpy(base.view(np.uint8).copy()).cuda()
    masters = torch.empty(M * SECTOR, dtype=torch.uint8, device="cuda")
    mplan.masters_device(masters.data_ptr(), base_d.data_ptr())
    torch.cuda.synchronize()
    files = file_descriptors(masters.data_ptr(), base, file_nsect)
    times = []
    for k in range(reps + 1):
        t0 = time.perf_counter()
        m = cv.master_build(files)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        info = m.info()
        m.close()
        if k:
            times.append(dt)
    best = min(times)
    return {"workload": f"sweep master set: {M} sectors in {file_nsect.size} device-resident files", "build_s": times,
            "sectors_per_s": M / best, "master_GBps": M * SECTOR / best / 1e9, "n_slots": info["n_slots"],
            "max_probe": info["max_probe"]}


def run_sweep(torch, cv, synth, stream, steps, sizes=(10**3, 10**5, 10**6, 10**7, 5 * 10**7),
              densities=(1e-4, 1e-2, 1e-1)):
    """Table-scaling sweep: an 8 GiB image (16,777,216 sectors, seed 3) against master sets of
    10^3 .. 5x10^7 sectors, with clusters planted at 0.01%, 1% and 10% of the image sectors
    (repeats allowed), scanned with and without the Bloom filter. Every result is checked
    against the plant log in full."""
    S = 16777216
    out = {"workload": "sweep: 8 GiB image, seed 3; master sets of the scale workload's size mix"}
    for M in sizes:
        file_nsect, mseed = synth.sweep_master_set(M)
        mplan = synth.Plan(0, mseed, 0, file_nsect, np.zeros(0, np.int32), np.zeros(0, np.uint32),
                           np.zeros(0, np.uint8))
        base = mplan.file_base()
        base_d = torch.from_numpy(base.view(np.uint8).copy()).cuda()
        masters = torch.empty(M * SECTOR, dtype=torch.uint8, device="cuda")
        mplan.masters_device(masters.data_ptr(), base_d.data_ptr())
        torch.cuda.synchronize()
        files = file_descriptors(masters.data_ptr(), base, file_nsect)
        t0 = time.perf_counter()
        tables = {"bloom": cv.master_build(files)}
        build_s = time.perf_counter() - t0
        tables["nobloom"] = cv.master_build(files, bloom_bits_per_key=0)
        del masters, base_d
        torch.cuda.synchronize()
        info = tables["bloom"].info()
        for dens in densities:
            plan = synth.make_plan_density(3, S, file_nsect, dens, mseed)
            image = image_on_device(torch, synth, plan)
            exp = plan.expected_intact()
            for name, m in tables.items():
                wall, kms, matches = time_scans(torch, cv, m, image, stream, steps)
                r = cv.scan(m, [image], stream=stream)
                exact = bool(np.array_equal(r.matches(0), exp))
                r.close()
                pr = cv.probe_profile(m, image, stream=stream)
                out[f"M{M}_d{dens:g}_{name}"] = {
                    "master_sectors": M, "files": int(file_nsect.size), "density": dens, "bloom": name == "bloom",
                    "table_MB": info["n_slots"] * 32 / 1e6, "bloom_MB": info["bloom_bytes"] / 1e6 if name == "bloom" else 0,
                    "max_probe": info["max_probe"], "build_s": build_s, "GBps": plan.n_bytes / wall / 1e9,
                    "kernel_GBps": plan.n_bytes / (kms * 1e-3) / 1e9, "kernel_ns_per_sector": kms * 1e6 / S,
                    "matches": matches, "exact_vs_plant_log": exact,
                    "bloom_pass_per_sector": pr["bloom_passed"] / S, "slot_reads_per_sector": pr["slot_reads"] / S,
                    "slot_reads_per_lookup": pr["slot_reads"] / max(pr["bloom_passed"], 1),
                    "found_sectors": pr["found"]}
            del image
            torch.cuda.synchronize()
        for m in tables.values():
            m.close()
    return out


def run_probe_profile(torch, cv, synth, sizes, image_gib, reps, density=0.01):
    """cv_probe_profile on an image of image_gib GiB (seed 3, clusters planted at `density`)
    against the sweep's master sets of each size, one table at a time (Bloom filter of 16 bits per
    key, then none), reps launches each: the exact table reads of the scan's lookups, for an ncu
    capture of probe_profile_kernel (L2 hit rate and DRAM bytes of the probes). Only the table,
    its filter, the image and the key words are on the device while the kernel runs."""
    S = (image_gib << 30) // SECTOR
    out = {"workload": f"{image_gib} GiB image (seed 3, {density:.0%} of clusters planted), sweep master sets",
           "reps": reps}
    for M in sizes:
        file_nsect, mseed = synth.sweep_master_set(M)
        mplan = synth.Plan(0, mseed, 0, file_nsect, np.zeros(0, np.int32), np.zeros(0, np.uint32), np.zeros(0, np.uint8))
        plan = synth.make_plan_density(3, S, file_nsect, density, mseed)
        image = image_on_device(torch, synth, plan)
        for bits in (16, 0):
            base = mplan.file_base()
            base_d = torch.from_numpy(base.view(np.uint8).copy()).cuda()
            masters = torch.empty(M * SECTOR, dtype=torch.uint8, device="cuda")
            mplan.masters_device(masters.data_ptr(), base_d.data_ptr())
            torch.cuda.synchronize()
            m = cv.master_build(file_descriptors(masters.data_ptr(), base, file_nsect), bloom_bits_per_key=bits)
            del masters, base_d
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            info = m.info()
            pr = None
            for _ in range(reps):
                pr = cv.probe_profile(m, image)
            out[f"M{M}_{'bloom' if bits else 'nobloom'}"] = {
                "master_sectors": M, "n_slots": info["n_slots"], "table_MB": info["n_slots"] * 32 / 1e6,
                "bloom_MB": info["bloom_bytes"] / 1e6, "sectors": pr["sectors"], "bloom_passed": pr["bloom_passed"],
                "slot_reads": pr["slot_reads"], "found": pr["found"],
                "l2_sector_requests_of_lookups": (pr["sectors"] if bits else 0) + pr["slot_reads"],
                "key_word_sector_requests": pr["sectors"] // 2}
            m.close()
            torch.cuda.synchronize()
        del image
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


# Algorithmic integer ops per 64-byte window: the rolled djb2 step with its key mix and filter
# tests; MD5 of one 64-byte message (a data block of 64 five-op steps, the padding block of 64
# four-op steps, two feed-forwards), or of the data block alone without padding.
FRAG_OPS_PER_WINDOW = {2: 31, 1: 64 * 5 + 4, 0: 64 * 5 + 64 * 4 + 8}


def run_fragments(torch, cv, synth, stream, steps, cpu_sample_bytes, config="frag", sigs=(2, 1, 0), sm_mhz=2070.0):
    """Section 5's fragment scan on the 4 GiB fragment workload: every 64-byte window at a 4-byte
    offset against the 64-byte fragments of 2,000 logos, for djb2-64 (rolled, confirmed), MD5
    without padding and MD5, each checked against the plant log."""
    import oracle

    fp = synth.frag_config(config)
    image = torch.empty(fp.n_bytes, dtype=torch.uint8, device="cuda")
    fp.image_device(torch, image)
    logos = fp.logos()
    exp = fp.expected_planted()
    windows = (fp.n_bytes - 64) // 4 + 1
    out = {"workload": "%s: %d-byte image, %d logos of log-uniform 1-16 KiB (%d fragments), half planted "
                       "1-3 times at 4-byte-aligned offsets" % (config, fp.n_bytes, fp.n_logos,
                                                               sum(x.size // 64 for x in logos)),
           "windows": windows}
    names = {2: "djb2_64", 1: "md5_nopad", 0: "md5"}
    for sig in sigs:
        name = names[sig]
        m = cv.master_build(logos, signature=sig, unit=cv.CV_UNIT_FRAGMENT)
        n_steps = steps if sig == 2 else max(2, steps // 5)
        wall, kms, matches = time_scans(torch, cv, m, image, stream, n_steps)
        r = cv.scan(m, [image], stream=stream)
        got = r.matches(0)
        r.close()
        planted_found = bool(np.isin(exp.view(np.dtype((np.void, 16))), got.view(np.dtype((np.void, 16)))).all())
        out[name] = {"GBps": fp.n_bytes / wall / 1e9, "count_kernel_GBps": fp.n_bytes / (kms * 1e-3) / 1e9,
                     "windows_per_s": windows / wall, "matches": matches, "planted_triples": int(exp.size),
                     "all_planted_found": planted_found}
        ops = FRAG_OPS_PER_WINDOW[sig]
        peak = SM_COUNT * INT_LANES_PER_SM_CLK * sm_mhz * 1e6
        achieved = windows * ops / (kms * 1e-3)
        hbm = measured_peaks().get("hbm_gbs", 6800.0)
        out[name]["roofline"] = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Top/s",
                                 "frac": achieved / peak, "ops_per_window": ops,
                                 "frac_of_hbm": out[name]["count_kernel_GBps"] / hbm,
                                 "peak_note": f"152 SMs x 128 int ops/clk x {sm_mhz:.0f} MHz"}
        m.close()
    if not cpu_sample_bytes:
        return out
    # the oracle on a bounded sample of the same image (all host cores)
    sample = image[:cpu_sample_bytes].cpu().numpy()
    t0 = time.perf_counter()
    oracle.frag_match(sample, logos)
    dt = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": sample.size / dt / 1e9, "unit": "GB/s", "cores": oracle.threads(), "kind": "oracle",
                           "sample": f"the first {sample.size >> 20} MiB of the image"}
    del image
    torch.cuda.synchronize()
    return out


def run_batched(torch, cv, synth, args, stream):
    """512 device images of uneven sizes (one device arena) against one 8M-sector table: one CUDA
    graph launch per run, autotuned, against 512 sequential cv_scan calls on the same images."""
    m, file_nsect, mseed, build_s = build_master_set(torch, cv, synth, "m8m")
    sizes = synth.batch_sizes(4, args.batch_images, 1 << 20, 2 << 30, args.batch_total_gib << 30)
    total = int(sizes.sum())
    arena = torch.empty(total * SECTOR, dtype=torch.uint8, device="cuda")
    images, expects, off = [], [], 0
    for i, n in enumerate(sizes.tolist()):
        plan = synth.make_plan_density(1000 + i, n, file_nsect, args.batch_density, mseed)
        ptrs, keep = device_plan(torch, synth, plan)
        plan.image_device(arena.data_ptr() + off * SECTOR, dev_plan=ptrs)
        if i % 64 == 0:
            torch.cuda.synchronize()
        expects.append(plan.expected_intact())
        images.append((arena.data_ptr() + off * SECTOR, n * SECTOR))
        off += n
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = cv.batch_create(m, images, autotune=True, stream=stream)
    tune_s = time.perf_counter() - t0
    info = b.info()
    for _ in range(3):
        b.run(stream)
        b.wait()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.batch_runs):
        b.run(stream)
    e1.record(stream)
    n_match = b.wait()
    graph_ms = e0.elapsed_time(e1) / args.batch_runs
    scan_ms = b.info()["scan_ms"]  # the scan launch of the last run, inside the graph
    exact = n_match == sum(e.size for e in expects)
    for i in range(0, len(images), max(1, len(images) // 16)):
        exact = exact and np.array_equal(cv.device_matches_to_numpy(b.matches(i)), expects[i])
    # the same images as 512 sequential plain scans
    seq = []
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for im in images:
            cv.scan(m, [im], keep_on_device=True, stream=stream).close()
        torch.cuda.synchronize()
        seq.append(time.perf_counter() - t0)
    seq_s = min(seq)
    b.close()
    m.close()
    tuned_by_occupancy = run_batch_tuner_occupancy(torch, cv, synth, images, expects, stream, file_nsect, mseed,
                                                   args.batch_runs)
    del arena
    torch.cuda.synchronize()
    return {"tuner_by_occupancy": tuned_by_occupancy,
            "workload": f"{len(images)} images, {total * SECTOR / 2**30:.0f} GiB, log-uniform 1 MiB-2 GiB scaled, "
                        f"{args.batch_density:.0%} of clusters planted from a {int(file_nsect.sum())}-sector table",
            "graph_GBps": total * SECTOR / (graph_ms * 1e-3) / 1e9, "graph_ms_per_run": graph_ms,
            "scan_launch_ms": scan_ms, "scan_launch_GBps": total * SECTOR / (scan_ms * 1e-3) / 1e9 if scan_ms else None,
            "sequential_GBps": total * SECTOR / seq_s / 1e9, "sequential_ms": seq_s * 1e3,
            "speedup_vs_sequential": (seq_s * 1e3) / graph_ms, "kernel_config": info["config_name"],
            "bloom": info["bloom"], "tuned": info["tuned"], "tune_s": tune_s, "kernel_nodes": info["kernel_launches"],
            "tensor_maps": info["tensor_maps"], "matches": n_match, "bit_exact_vs_plant_log": bool(exact),
            "table_build_s": build_s}


def run_streamed(torch, cv, synth, scale_plan, master, pool, stream, total_gib, link_gbps, chunk_gib=1):
    """The streamed variant of the scale workload: a distinct image (seed 2) of total_gib GiB in
    pinned host memory, fed to cv_scan in 1 GiB chunks. The image never exists whole: a generator
    thread (the host generator, OpenMP over all cores) writes chunk c into slot c mod P of the
    pinned pool (P = the pool's size in chunks) once the scan of chunk c - P has returned, and the
    main thread scans every chunk that has landed, several per call when they are ready (the
    library copies them to the device through its ring, copies overlapping the hashing). Every
    chunk's matches are checked against the plan's plant log."""
    import threading

    chunk_s = (chunk_gib << 30) // SECTOR
    n_chunks = (total_gib << 30) // (chunk_gib << 30)
    slots = max(2, pool.numel() // (chunk_gib << 30))
    plan = synth.make_plan(2, n_chunks * chunk_s, scale_plan.file_nsect, 0.25, master_seed=scale_plan.master_seed)
    expect = plan.expected_intact()
    base = pool.data_ptr()
    ready = [threading.Event() for _ in range(n_chunks)]
    free = [threading.Semaphore(1) for _ in range(slots)]
    gen_s = [0.0]

    def generator():
        for c in range(n_chunks):
            free[c % slots].acquire()
            t0 = time.perf_counter()
            plan.image_host_into(base + (c % slots) * (chunk_gib << 30), c * chunk_s, chunk_s)
            gen_s[0] += time.perf_counter() - t0
            ready[c].set()

    th = threading.Thread(target=generator, daemon=True)
    exact, matches, kernel_ms, calls = True, 0, 0.0, 0
    t0 = time.perf_counter()
    th.start()
    c = 0
    while c < n_chunks:
        ready[c].wait()
        batch = [c]
        while batch[-1] + 1 < n_chunks and len(batch) < slots // 2 and ready[batch[-1] + 1].is_set():
            batch.append(batch[-1] + 1)
        imgs = [(base + (k % slots) * (chunk_gib << 30), chunk_gib << 30) for k in batch]
        r = cv.scan(master, imgs, chunk_bytes=chunk_gib << 30, stream=stream)
        st = r.stats()
        kernel_ms += st["kernel_ms"]
        matches += st["matches"]
        for j, k in enumerate(batch):
            if not np.array_equal(r.matches(j), expected_window(expect, k * chunk_s, chunk_s)):
                exact = False
        r.close()
        calls += 1
        for k in batch:
            free[k % slots].release()
        c = batch[-1] + 1
    th.join()
    wall = time.perf_counter() - t0
    nbytes = n_chunks * (chunk_gib << 30)
    gen_gbps = nbytes / gen_s[0] / 1e9
    return {"workload": f"seed-2 image of {total_gib} GiB ({n_chunks * chunk_s} sectors), generated chunk by chunk "
                        f"into a {slots * chunk_gib} GiB pinned pool, scanned in {chunk_gib} GiB chunks against the "
                        f"scale workload's {scale_plan.n_master_sectors}-sector table",
            "GBps": nbytes / wall / 1e9, "seconds": wall, "scan_calls": calls,
            "kernel_GBps": nbytes / (kernel_ms * 1e-3) / 1e9, "generator_GBps": gen_gbps,
            "h2d_link_GBps": link_gbps, "bound": "host generator" if gen_gbps < link_gbps else "host-to-device copies",
            "matches": matches, "planted_matches": int(expect.size), "bit_exact_vs_plant_log": bool(exact)}


def run_batch_tuner_occupancy(torch, cv, synth, images, expects, stream, file_nsect, mseed, runs,
                              occupancies=(0.5, 0.9)):
    """The batch tuner on masters without a Bloom filter at a given occupancy (a prefix of the
    8M-sector master set in a 2^23-slot hash table): what it picks among configuration x layout
    (the hash table, or a sorted copy) x Bloom (off, or a filter the batch builds), how fast the
    choice scans, and its result against the plant log (matches of the prefix's files)."""
    base = np.zeros(file_nsect.size + 1, np.uint64)
    np.cumsum(file_nsect, dtype=np.uint64, out=base[1:])
    cum = base[1:].astype(np.int64)
    slots = 1 << 23
    masters = torch.empty(int(base[-1]) * SECTOR, dtype=torch.uint8, device="cuda")
    mplan = synth.Plan(0, mseed, 0, file_nsect, np.zeros(0, np.int32), np.zeros(0, np.uint32), np.zeros(0, np.uint8))
    base_d = torch.from_numpy(base.view(np.uint8).copy()).cuda()
    mplan.masters_device(masters.data_ptr(), base_d.data_ptr())
    torch.cuda.synchronize()
    out = {}
    for occ in occupancies:
        k = max(int(np.searchsorted(cum, occ * (slots - 1) * 0.999, side="right")), 1)
        files = file_descriptors(masters.data_ptr(), base, file_nsect)[:k]
        max_load = min(0.9, float(cum[k - 1]) / (slots * 0.9999))
        m = cv.master_build(files, max_load=max_load, bloom_bits_per_key=0)
        info_m = m.info()
        t0 = time.perf_counter()
        b = cv.batch_create(m, images, autotune=True, stream=stream)
        tune_s = time.perf_counter() - t0
        info = b.info()
        b.run(stream)
        b.wait()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(runs):
            b.run(stream)
        e1.record(stream)
        n_match = b.wait()
        ms = e0.elapsed_time(e1) / runs
        want = [e[e["file_id"] < k] for e in expects]
        exact = n_match == sum(w.size for w in want)
        for i in range(0, len(images), max(1, len(images) // 16)):
            exact = exact and np.array_equal(cv.device_matches_to_numpy(b.matches(i)), want[i])
        total = sum(nb for _, nb in images)
        out[f"occupancy_{occ:g}"] = {
            "master_sectors": int(cum[k - 1]), "occupancy": info_m["n_unique"] / info_m["n_slots"],
            "chosen_config": info["config_name"], "chosen_layout": "sorted" if info["layout"] else "hash",
            "chosen_bloom": bool(info["bloom"]), "graph_GBps": total / (ms * 1e-3) / 1e9, "tune_s": tune_s,
            "bit_exact_vs_plant_log": bool(exact)}
        b.close()
        m.close()
    del masters
    torch.cuda.synchronize()
    return out


def h2d_link_gbps(torch, host, stream, nbytes=8 << 30):
    """One plain host-to-device copy of nbytes of the pinned buffer, timed with CUDA events."""
    probe = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    probe.copy_(host[:nbytes], non_blocking=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    del probe
    return nbytes / (ev0.elapsed_time(ev1) * 1e-3) / 1e9


def run_served(torch, cv, synth, args, host, rate=None, n_requests=None):
    """Poisson arrivals of host-resident requests (80% 64 KiB-4 MiB stream chunks, 20%
    256 MiB-16 GiB drive images, windows of one pinned pool) against one 8M-sector table. The
    host link is timed right before and after the run (a plain 8 GiB copy from the pool)."""
    import threading

    rate = rate or args.serve_rate
    m, file_nsect, mseed, build_s = build_master_set(torch, cv, synth, "m8m")
    pool_sectors = host.numel() // SECTOR
    plan = synth.make_plan_density(5, pool_sectors, file_nsect, args.serve_density, mseed)
    ptrs, keep = device_plan(torch, synth, plan)
    pool = torch.empty(pool_sectors * SECTOR, dtype=torch.uint8, device="cuda")
    plan.image_device(pool.data_ptr(), dev_plan=ptrs)
    host.copy_(pool)
    del pool, keep
    torch.cuda.synchronize()
    expect = plan.expected_intact()
    rng = np.random.default_rng(5)
    n = n_requests or args.serve_requests
    gaps = rng.exponential(1.0 / rate, size=n)
    drive = rng.random(n) < 0.2
    size_b = np.where(drive, np.exp(rng.uniform(np.log(256 << 20), np.log(16 << 30), n)),
                      np.exp(rng.uniform(np.log(64 << 10), np.log(4 << 20), n)))
    size_s = np.maximum((size_b // 4096).astype(np.int64), 1) * 8
    size_s = np.minimum(size_s, pool_sectors // 8 * 8)
    start = (rng.integers(0, (pool_sectors - size_s) // 8 + 1) * 8).astype(np.int64)
    srv = cv.server_create(m, hbm_budget_bytes=args.serve_budget_gb * 10**9, work_unit_bytes=64 << 20, max_live=64,
                           copy_streams=4, max_copy_bytes=int(args.serve_copy_gib * 2**30) if args.serve_copy_gib else 0)
    base = host.data_ptr()
    tickets = [None] * n
    arrivals = np.cumsum(gaps)

    def submitter():
        t0 = time.perf_counter()
        for k in range(n):
            wait = arrivals[k] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets[k] = srv.submit((base + int(start[k]) * SECTOR, int(size_s[k]) * SECTOR), tag=k)

    link_before = h2d_link_gbps(torch, host, torch.cuda.current_stream())
    th = threading.Thread(target=submitter)
    t0 = time.perf_counter()
    th.start()
    exact = True
    lat = np.zeros(n)
    for k in range(n):
        while tickets[k] is None:
            time.sleep(0.0005)
        r = srv.poll(tickets[k], timeout_ms=-1)
        got = r.matches(0)
        lat[k] = r.stats()["total_ms"]
        r.close()
        if not np.array_equal(got, expected_window(expect, int(start[k]), int(size_s[k]))):
            exact = False
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    m.close()
    link_after = h2d_link_gbps(torch, host, torch.cuda.current_stream())
    total_b = int(size_s.sum()) * SECTOR
    return {"workload": f"{n} requests, Poisson {rate:g}/s, 80% 64 KiB-4 MiB / 20% 256 MiB-16 GiB, "
                        f"windows of a {pool_sectors * SECTOR / 2**30:.0f} GiB pinned pool, "
                        f"{int(file_nsect.sum())}-sector table, HBM budget {args.serve_budget_gb} GB",
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
            "chunks_p50_ms": float(np.percentile(lat[~drive], 50)), "chunks_p99_ms": float(np.percentile(lat[~drive], 99)),
            "drives_p50_ms": float(np.percentile(lat[drive], 50)), "drives_p99_ms": float(np.percentile(lat[drive], 99)),
            "drives_copy_floor_p99_ms": float(np.percentile(size_s[drive] * SECTOR / (args.h2d_link_gbps * 1e9) * 1e3,
                                                            99)),
            "h2d_link_GBps_before": link_before, "h2d_link_GBps_after": link_after,
            "offered_GBps": float(size_s.mean()) * SECTOR * rate / 1e9,
            "littles_law_mean_live": rate * st["mean_ms"] * 1e-3,
            "host_memory": "cudaHostAlloc (torch pin_memory)",
            "throughput_GBps": total_b / st["wall_s"] / 1e9 if st["wall_s"] else None, "wall_s": wall,
            "bytes": total_b, "iterations": st["iterations"], "units": st["units"],
            "units_per_scan_launch": st["units"] / max(st["iterations"], 1),
            "mean_live_per_iteration": st["mean_live_per_iteration"],
            "peak_bytes_in_flight": st["peak_bytes_in_flight"], "completed": st["completed"], "failed": st["failed"],
            "bit_exact_vs_plant_log": bool(exact)}


METRIC = "disk-image GB/s scanned on 1 GB300 (% of hash/HBM roofline); p99 scan latency served"


def emit_section(args, name, obj):
    """One section of the results as its own JSON line on stdout (rank 0), ahead of the headline
    line, which comes last and stays short; also appended to --sections-out when given."""
    if int(os.environ.get("RANK", "0")) != 0 or obj is None:
        return
    text = json.dumps({"section": name, **obj}, separators=(",", ":"))
    print(text, flush=True)
    if args.sections_out:
        with open(args.sections_out, "a") as fh:
            fh.write(text + "\n")


def scan_roofline(kms, sectors, hit_sectors, clocks, int_peak, args):
    """The scan kernel against the lower of its two ceilings.

    Algorithmic bytes per launch: the image read once (512 B per sector), one 16-byte hit record
    per sector with a match, and the per-tile counts (4 + 8 B per 32-sector output tile). The
    integer ceiling is 152 SMs x 128 lanes x the sampled SM clock, at 2,852 algorithmic MD5 ops
    per sector (5.57 per byte); the HBM ceiling is the measured copy bandwidth. The lower one is
    the bound reported."""
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    hbm = measured_peaks().get("hbm_gbs")
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)"
    if not hbm:
        hbm, hbm_src = 6800.0, "fallback"
    peak_ops = SM_COUNT * INT_LANES_PER_SM_CLK * sm_mhz * 1e6
    int_roof_gbs = peak_ops / (MD5_OPS_PER_SECTOR / SECTOR) / 1e9
    alg_bytes = sectors * SECTOR + hit_sectors * 16 + (sectors + 31) // 32 * 12
    achieved_gbs = alg_bytes / (kms * 1e-3) / 1e9
    achieved_ops = sectors * MD5_OPS_PER_SECTOR / (kms * 1e-3)
    traffic = SCAN_TRAFFIC_BYTES.get(args.config) if args.kernel_config == 0 and not args.signature else None
    if hbm <= int_roof_gbs:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm}
    else:
        roof = {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12, "unit": "Top/s",
                "frac": achieved_ops / peak_ops}
    roof.update({
        "traffic": traffic, "kernel": "scan_kernel (MD5 + Bloom + probe + tile compaction)", "kernel_ms": kms,
        "peak_source": hbm_src, "int_roof_GBps": int_roof_gbs,
        "alu_frac_of_issue_ceiling": achieved_ops / peak_ops,
        "alu_frac_of_measured_int_peak": achieved_ops / (int_peak["mixed_ops_per_s"] * 1e12),
        "detail": {
            "algorithmic_bytes_per_launch": alg_bytes, "kernel_GBps_image": sectors * SECTOR / (kms * 1e-3) / 1e9,
            "achieved_int_Tops": achieved_ops / 1e12, "issue_ceiling_Tops": peak_ops / 1e12,
            "int_peak_measured": int_peak, "hash_hbm_roofline_GBps": min(hbm, int_roof_gbs),
            "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum per launch, from one ncu capture of the "
                            "same kernel on the 4 GiB mid workload (4.3773 GB), scaled x8 by sectors to the 32 GiB "
                            "image",
            "peak_note": f"{SM_COUNT} SMs x {INT_LANES_PER_SM_CLK} int ops/clk x median SM clock {sm_mhz:.0f} MHz "
                         f"sampled in the timed region; {MD5_OPS_PER_SECTOR} algorithmic ops per sector"}})
    return roof


def headline(*, value, world, args, ms, nbytes, sectors, plan, kernel_config, matches, exact, roof, clocks, e2e,
             cpu, launches, batched, served):
    """The last stdout line: the headline figures only (the sections went out on earlier lines)."""
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic (seeded generator, the paper's random-file workload mix)",
        "config": {"workload": f"{args.config}: {nbytes / 2**30:.0f} GiB image ({sectors} sectors), "
                               f"{plan.n_master_sectors} master sectors in {plan.n_files} files, MD5, device-resident",
                   "l2": "inputs larger than L2 (no flush)", "kernel_config": kernel_config,
                   "matches_per_step": matches, "bit_exact_vs_plant_log": exact},
        "sectors_per_s": world * sectors / (ms * 1e-3),
        "roofline": roof,
        "clocks": {k: clocks.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples")},
        "e2e": None if e2e is None else {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step",
                                                              "d2h_bytes_per_step", "frac_of_h2d_link")},
        "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "gpu_launches": launches,
    }
    if batched:
        line["batched"] = {"GBps": batched["graph_GBps"], "speedup_vs_sequential": batched["speedup_vs_sequential"],
                           "bit_exact": batched["bit_exact_vs_plant_log"]}
    if served:
        line["served"] = {"p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"],
                          "GBps": served["throughput_GBps"], "bit_exact": served["bit_exact_vs_plant_log"]}
        line["p99_served_ms"] = served["p99_ms"]
    line["sections"] = "earlier stdout lines, one JSON object each, keyed by 'section'"
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="scale")
    ap.add_argument("--kernel-config", type=int, default=0)
    ap.add_argument("--signature", type=int, default=0,
                    help="signature of the main scan's table (0 MD5, the headline; 1-3 for profiling runs)")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-streamed", action="store_true", help="skip the streamed variant of e2e")
    ap.add_argument("--streamed-gib", type=int, default=128, help="size of the streamed variant's image")
    ap.add_argument("--cpu-sample-pieces", type=int, default=24, help="1 GiB pieces timed on the oracle")
    ap.add_argument("--ref-sample-sectors", type=int, default=1 << 19)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-sigs", action="store_true")
    ap.add_argument("--sig-steps", type=int, default=20)
    ap.add_argument("--no-tables", action="store_true")
    ap.add_argument("--no-frag", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=5)
    ap.add_argument("--sweep-only", action="store_true", help="run only the table-scaling sweep and print its JSON")
    ap.add_argument("--build-only", type=int, default=0, metavar="M",
                    help="time only table builds of the sweep's master set of M sectors and print their JSON")
    ap.add_argument("--probe-only", default="", metavar="M,M,...",
                    help="run only cv_probe_profile against the sweep's master sets of these sizes and print JSON")
    ap.add_argument("--probe-gib", type=int, default=1)
    ap.add_argument("--probe-reps", type=int, default=2)
    ap.add_argument("--frag-steps", type=int, default=10)
    ap.add_argument("--frag-cpu-mib", type=int, default=256)
    ap.add_argument("--frag-only", action="store_true",
                    help="run only the fragment scan (--frag-config, --frag-sigs) and print its JSON")
    ap.add_argument("--frag-config", default="frag")
    ap.add_argument("--frag-sigs", default="2,1,0")
    ap.add_argument("--table-steps", type=int, default=10)
    ap.add_argument("--batch-images", type=int, default=512)
    ap.add_argument("--batch-total-gib", type=int, default=64)
    ap.add_argument("--batch-density", type=float, default=0.01)
    ap.add_argument("--batch-runs", type=int, default=10)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-density", type=float, default=0.02)
    ap.add_argument("--serve-budget-gb", type=int, default=120)
    ap.add_argument("--serve-copy-gib", type=float, default=0.0, help="copy bytes queued at once (0: the library's)")
    ap.add_argument("--h2d-link-gbps", type=float, default=211.0, help="host link rate for the drives' copy floor")
    ap.add_argument("--serve-only", action="store_true", help="run only the served section and print its JSON")
    ap.add_argument("--serve-rate-high", type=float, default=200.0,
                    help="a second served run at this arrival rate (0: none), to show continuous batching")
    ap.add_argument("--serve-requests-high", type=int, default=1000)
    ap.add_argument("--sections-out", default="", help="also append every section's JSON line to this file")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return run_reference(args)
    if args.serve_only:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        from paper_0901_1307_gb300 import cv, synth

        host = torch.empty(32 << 30, dtype=torch.uint8, pin_memory=True)
        print(json.dumps(run_served(torch, cv, synth, args, host)))
        return 0
    if args.build_only:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        from paper_0901_1307_gb300 import cv, synth

        print(json.dumps(run_build(torch, cv, synth, args.build_only)))
        return 0
    if args.probe_only:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        from paper_0901_1307_gb300 import cv, synth

        sizes = tuple(int(float(x)) for x in args.probe_only.split(","))
        print(json.dumps(run_probe_profile(torch, cv, synth, sizes, args.probe_gib, args.probe_reps)))
        return 0
    if args.sweep_only:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        from paper_0901_1307_gb300 import cv, synth

        print(json.dumps(run_sweep(torch, cv, synth, torch.cuda.current_stream(), args.sweep_steps)))
        return 0
    if args.frag_only:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        from paper_0901_1307_gb300 import cv, synth

        sigs = tuple(int(x) for x in args.frag_sigs.split(","))
        print(json.dumps(run_fragments(torch, cv, synth, torch.cuda.current_stream(), args.frag_steps,
                                       args.frag_cpu_mib << 20, args.frag_config, sigs)))
        return 0

    import torch

    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    from paper_0901_1307_gb300 import cv, synth

    plan, image, master, build_s = setup_workload(torch, cv, synth, args.config, seed_offset=1000 * rank,
                                                  signature=args.signature)
    stream = torch.cuda.current_stream()

    def step(buf, keep_on_device=True):
        r = cv.scan(master, [buf], keep_on_device=keep_on_device, stream=stream, kernel_config=args.kernel_config)
        return r

    for _ in range(args.warmup):
        step(image).close()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    kernel_ms, matches, launches, hit_sectors, used_config = [], 0, 0, 0, 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            r = step(image)
            st = r.stats()
            kernel_ms.append(st["kernel_ms"])
            matches = st["matches"]
            hit_sectors = st["hit_sectors"]
            used_config = st["kernel_config"]
            launches += st["kernel_launches"]
            r.close()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    clocks = clk.summary()
    nbytes = plan.n_bytes
    value = world * nbytes / (ms * 1e-3) / 1e9
    # the timed call's result at full size, against the plan's plant log (untimed)
    r = step(image, keep_on_device=False)
    exact = bool(np.array_equal(r.matches(0), plan.expected_intact()))
    r.close()

    if not args.no_sigs:
        emit_section(args, "signatures", run_signatures(torch, cv, synth, plan, image, stream, args.sig_steps))
    if not args.no_tables:
        emit_section(args, "tables", run_tables(torch, cv, synth, plan, image, stream, args.table_steps))

    # end to end through the C ABI from pinned host memory
    e2e = None
    host = None
    if not args.no_e2e or not args.no_serve:
        host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        host.copy_(image)
    del image
    torch.cuda.synchronize()
    if not args.no_e2e:
        # the host link itself, before and after the timed steps: one plain copy of 8 GiB of the
        # pinned image to the device
        link_before = h2d_link_gbps(torch, host, stream)
        for _ in range(2):
            step(host, keep_on_device=False).close()
        torch.cuda.synchronize()
        d2h, step_s = 0, []
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            r = step(host, keep_on_device=False)
            d2h = r.count(0) * 16
            r.close()
            step_s.append(time.perf_counter() - t1)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": world * nbytes / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps, "step_s": step_s}
        link = h2d_link_gbps(torch, host, stream)
        e2e["h2d_link_GBps_before"] = link_before
        e2e["h2d_link_GBps"] = link
        e2e["frac_of_h2d_link"] = e2e["value"] / world / max(link, link_before)
        if not args.no_streamed and rank == 0:  # host-bound and not part of the scaled metric
            e2e["streamed"] = run_streamed(torch, cv, synth, plan, master, host, stream, args.streamed_gib, link)

    if e2e is not None:
        emit_section(args, "e2e", e2e)

    if not args.no_sweep and rank == 0:
        emit_section(args, "table_sweep", run_sweep(torch, cv, synth, stream, args.sweep_steps))

    if not args.no_frag and rank == 0:
        emit_section(args, "fragments", run_fragments(
            torch, cv, synth, stream, args.frag_steps, args.frag_cpu_mib << 20, args.frag_config,
            tuple(int(x) for x in args.frag_sigs.split(",")), clocks.get("sm_mhz") or 2070.0))

    ip = cv.int_peak()
    int_peak = {k: ip[k] / 1e12 for k in ("alu_ops_per_s", "fma_ops_per_s", "mixed_ops_per_s")}
    int_peak.update({"unit": "Top/s", "sm_clock_mhz": ip["sm_clock_mhz"],
                     "mixed_ops_per_clk_per_sm": ip["mixed_ops_per_s"] / (ip["sms"] * ip["sm_clock_mhz"] * 1e6),
                     "how": "cv_int_peak: independent lop3 / mad.lo chains, 8 blocks of 256 threads per SM"})
    kms = statistics.mean(kernel_ms)
    sectors = plan.n_sectors
    roof = scan_roofline(kms, sectors, hit_sectors, clocks, int_peak, args)
    if args.signature:
        roof["kernel"] = f"scan_kernel with signature {args.signature} (profiling run; ops figures are MD5's)"
    emit_section(args, "roofline_detail", roof.pop("detail"))
    master.close()
    batched = served = None
    # the batched and served workloads are single-GPU configurations: rank 0 runs them
    if not args.no_batch and rank == 0:
        batched = run_batched(torch, cv, synth, args, stream)
        emit_section(args, "batched", batched)
    if not args.no_serve and rank == 0:
        # serving gets a pinned pool of its own, allocated here (the e2e buffer above was rewritten
        # by the host generator of the streamed variant)
        serve_host = torch.empty(host.numel(), dtype=torch.uint8, pin_memory=True)
        del host
        host = serve_host
        served = run_served(torch, cv, synth, args, host)
        emit_section(args, "served", served)
        if args.serve_rate_high:
            emit_section(args, "served_high_rate", run_served(torch, cv, synth, args, host, args.serve_rate_high,
                                                              args.serve_requests_high))
    del host
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(plan, args.cpu_sample_pieces)
        emit_section(args, "cpu_baseline", cpu)
    line = headline(value=value, world=world, args=args, ms=ms, nbytes=nbytes, sectors=sectors, plan=plan,
                    kernel_config=cv.kernel_configs()[used_config] + ("" if args.kernel_config else " (default)"),
                    matches=matches, exact=exact, roof=roof, clocks=clocks, e2e=e2e, cpu=cpu, launches=launches,
                    batched=batched, served=served)
    if rank == 0:
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
