"""GPU parity: the CUDA path through the C ABI against the CPU oracle, on the same seeded inputs.

Everything here is integer work, so the bar is bit-exact: identical digests, identical trivial
flags, identical sorted match lists.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_same(got, want, what=""):
    """Bit-exact comparison of two sorted triple arrays, naming the differences on failure."""
    if np.array_equal(got, want):
        return
    g = set(map(tuple, np.stack([got["disk_sector"], got["file_id"], got["file_sector"]], 1).tolist()))
    w = set(map(tuple, np.stack([want["disk_sector"], want["file_id"], want["file_sector"]], 1).tolist()))
    miss, extra = sorted(w - g), sorted(g - w)
    raise AssertionError(f"{what}: got {got.size} want {want.size}; missing {len(miss)} {miss[:16]}; "
                         f"extra {len(extra)} {extra[:16]}; order ok={sorted(g) == [tuple(x) for x in got.tolist()]}")


def gpu_digests(cv, img_t, n):
    out = torch.empty(max(n, 1) * 16, dtype=torch.uint8, device="cuda")
    triv = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    cv.sector_digests(img_t.data_ptr(), n, out.data_ptr(), triv.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()[: n * 16].reshape(n, 16), triv.cpu().numpy()[:n].astype(bool)


# ------------------------------------------------------------------------- digests


@pytest.mark.parametrize("n", [1, 31, 129, 1000, 65536 + 77])
def test_digests_every_sector_class(cv, n):
    plan = synth.config_plan("small:70000:30:11")
    img = plan.image_host(0, n)
    # add trivial and near-trivial sectors
    secs = img.reshape(n, SECTOR)
    for k in range(0, n, 97):
        secs[k] = k & 0xFF
    for k in range(5, n, 89):
        secs[k] = 0
        secs[k, 511] = 1
    d, t = gpu_digests(cv, dev(img), n)
    assert np.array_equal(d, oracle.md5_sectors(img))
    assert np.array_equal(t, np.array([oracle.sector_trivial(s) for s in secs]))


def test_digests_ten_million_sampled(cv):
    """10^7 random sectors generated on the device; 200k of them checked against the oracle."""
    plan = synth.make_plan(77, 10_000_000, [16], 0.0)
    n = plan.n_sectors
    img = torch.empty(n * SECTOR, dtype=torch.uint8, device="cuda")
    keep = _device_plan(plan)
    plan.image_device(img.data_ptr(), dev_plan=keep[0])
    out = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    cv.sector_digests(img.data_ptr(), n, out.data_ptr())
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    for start in rng.integers(0, n - 2000, size=100):
        host = plan.image_host(int(start), 2000)
        got = out[int(start) * 16:(int(start) + 2000) * 16].cpu().numpy().reshape(2000, 16)
        assert np.array_equal(got, oracle.md5_sectors(host))
    del img, out


def _device_plan(plan):
    """Device copies of the plan arrays (kept alive by the caller)."""
    pf = dev(plan.plant_file.view(np.uint8))
    pc = dev(plan.plant_fcluster.view(np.uint8))
    po = dev(plan.plant_over)
    fn = dev(plan.file_nsect.view(np.uint8))
    vc = dev(synth.vocab(plan.image_seed))
    return (pf.data_ptr(), pc.data_ptr(), po.data_ptr(), fn.data_ptr(), vc.data_ptr()), (pf, pc, po, fn, vc)


def test_device_generator_equals_host_generator(cv):
    plan = synth.config_plan("small:20000:40:5")
    ptrs, keep = _device_plan(plan)
    img = torch.empty(plan.n_bytes, dtype=torch.uint8, device="cuda")
    plan.image_device(img.data_ptr(), dev_plan=ptrs)
    torch.cuda.synchronize()
    assert np.array_equal(img.cpu().numpy(), plan.image_host())
    base = dev(plan.file_base().view(np.uint8))
    ms = torch.empty(plan.n_master_sectors * SECTOR, dtype=torch.uint8, device="cuda")
    plan.masters_device(ms.data_ptr(), base.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(ms.cpu().numpy(), np.concatenate(plan.masters_host()))


# ---------------------------------------------------------------------------- scan


def _tricky(seed):
    from test_oracle import tricky_case

    return tricky_case(seed)


@pytest.mark.parametrize("seed", range(6))
def test_scan_tricky_cases(cv, seed):
    image, files = _tricky(seed)
    want = oracle.match_brute(image, files)
    with cv.master_build(files) as m:
        with cv.scan(m, [dev(image)]) as r:
            assert_same(r.matches(0), want)
        with cv.scan(m, [image]) as r:  # host image, streamed
            assert_same(r.matches(0), want)


def test_scan_tiny_workload_full(cv):
    """The 64 MiB workload in full: GPU == oracle == plant log."""
    plan = synth.config_plan("tiny")
    img = plan.image_host()
    files = plan.masters_host()
    want = oracle.match_hash(img, files)
    assert np.array_equal(want, plan.expected_intact())
    with cv.master_build(files) as m:
        info = m.info()
        assert info["n_kept"] == plan.n_master_sectors and info["n_unique"] == plan.n_master_sectors
        with cv.scan(m, [dev(img)]) as r:
            assert_same(r.matches(0), want)
        with cv.scan(m, [img], chunk_bytes=3 * 1024 * 1024 + 512) as r:  # 22 ragged chunks
            assert_same(r.matches(0), want)


@pytest.mark.parametrize("cfg_k", range(5))
def test_every_kernel_config_same_result(cv, cfg_k):
    names = cv.kernel_configs()
    if cfg_k >= len(names):
        pytest.skip("no such configuration")
    plan = synth.config_plan("small:50001:60:9")  # ragged: not a multiple of any tile
    img = plan.image_host()
    files = plan.masters_host()
    want = oracle.match_hash(img, files)
    with cv.master_build(files) as m, cv.scan(m, [dev(img)], kernel_config=cfg_k + 1) as r:
        assert_same(r.matches(0), want, names[cfg_k])


@pytest.mark.parametrize("max_load,bloom", [(0.5, 0), (0.9, 0xFFFFFFFF), (0.25, 8), (0.9, 0)])
def test_table_options_do_not_change_result(cv, max_load, bloom):
    plan = synth.config_plan("small:40000:80:13")
    img = plan.image_host()
    files = plan.masters_host()
    # duplicates across files: copy some sectors of file 0 into file 1
    files[1][:4 * SECTOR] = files[0][:4 * SECTOR]
    want = oracle.match_hash(img, files)
    with cv.master_build(files, max_load=max_load, bloom_bits_per_key=bloom) as m:
        with cv.scan(m, [dev(img)]) as r:
            assert_same(r.matches(0), want)


def test_many_images_uneven_sizes(cv):
    plan = synth.config_plan("small:30000:40:17")
    files = plan.masters_host()
    full = plan.image_host()
    cuts = [(0, 0), (0, 100), (100, 5000 * SECTOR + 300), (7000 * SECTOR, 7001 * SECTOR),
            (8000 * SECTOR, 30000 * SECTOR), (12345 * SECTOR + 7, 12345 * SECTOR + 7 + 512 * 9)]
    images, wants = [], []
    for k, (a, b) in enumerate(cuts):
        piece = np.ascontiguousarray(full[a:b])
        wants.append(oracle.match_hash(piece, files))
        if a % 16 == 0 and k % 2 == 0:
            images.append(dev(piece))
        else:
            images.append(piece)  # host buffers, also the misaligned one
    with cv.master_build(files) as m, cv.scan(m, images) as r:
        for k in range(len(cuts)):
            assert_same(r.matches(k), wants[k], str(k))


def test_empty_master_set_and_trivial_only(cv):
    img = synth.random_sectors(5, 300)
    with cv.master_build([]) as m, cv.scan(m, [dev(img)]) as r:
        assert r.count(0) == 0
    zeros = np.zeros(16 * SECTOR, np.uint8)
    fills = np.full(16 * SECTOR, 0x41, np.uint8)
    img2 = np.concatenate([zeros, fills, img])
    with cv.master_build([zeros, fills]) as m:
        assert m.info()["n_kept"] == 0
        with cv.scan(m, [dev(img2)]) as r:
            assert r.count(0) == 0


def test_misaligned_device_image_rejected(cv):
    img = dev(synth.random_sectors(1, 8))
    with cv.master_build([synth.random_sectors(2, 4)]) as m:
        with pytest.raises(cv.CVError) as e:
            cv.scan(m, [(img.data_ptr() + 4, 4 * SECTOR)])
        assert e.value.code == cv.CV_EINVAL


def test_keep_on_device(cv):
    plan = synth.config_plan("small:20000:30:19")
    img = plan.image_host()
    files = plan.masters_host()
    want = oracle.match_hash(img, files)
    with cv.master_build(files) as m, cv.scan(m, [dev(img)], keep_on_device=True) as r:
        dm = r.matches(0)
        t = torch.as_tensor(dm, device="cuda").cpu().numpy()
        got = np.zeros(t.shape[0], oracle.TRIPLE_DTYPE)
        got["disk_sector"] = t[:, 0]
        got["file_id"] = t[:, 1] & 0xFFFFFFFF
        got["file_sector"] = t[:, 1] >> 32
        assert np.array_equal(got, want)


def test_images_sharing_one_allocation(cv):
    """Images carved out of one device buffer: sector-aligned ones share a tensor map over the
    whole allocation, a 16-byte-aligned one gets its own; results equal separate scans."""
    plan = synth.config_plan("small:60000:50:23")
    files = plan.masters_host()
    full = plan.image_host()
    whole = dev(full)
    cuts = [(0, 7000), (7000, 7003), (7003, 31000), (31000, 31000), (40000, 60000)]
    images, wants = [], []
    for a, b in cuts:
        images.append((whole.data_ptr() + a * SECTOR, (b - a) * SECTOR))
        wants.append(oracle.match_hash(full[a * SECTOR:b * SECTOR], files))
    off = 12345 * SECTOR + 16  # 16-byte aligned, not sector-aligned within the allocation
    images.append((whole.data_ptr() + off, 9000 * SECTOR))
    wants.append(oracle.match_hash(full[off:off + 9000 * SECTOR], files))
    with cv.master_build(files) as m, cv.scan(m, images) as r:
        for k in range(len(images)):
            assert_same(r.matches(k), wants[k], str(k))


def test_many_segments_and_launches_every_config(cv):
    """450 images in one scan: 300 of 0-39 sectors carved from one buffer (many segments, most
    smaller than a tile, so a block's consecutive tiles keep changing segment) and 150 of 1-199
    sectors, each 16 bytes into a buffer of its own so that each needs its own tensor map (more
    than one launch carries), interleaved. Every configuration, against the oracle's result for
    the whole image cut per image (each sector is matched on its own)."""
    plan = synth.config_plan("small:40000:60:61")
    full = plan.image_host()
    files = plan.masters_host()
    want_all = oracle.match_hash(full, files)

    def want(a, n):
        sel = want_all[(want_all["disk_sector"] >= a) & (want_all["disk_sector"] < a + n)].copy()
        sel["disk_sector"] -= a
        return sel

    rng = np.random.default_rng(61)
    whole = dev(full)
    images, wants, keep = [], [], []
    a = 0
    for _ in range(300):
        n = int(rng.integers(0, 40))
        images.append((whole.data_ptr() + a * SECTOR, n * SECTOR))
        wants.append(want(a, n))
        a += n
    for _ in range(150):
        n = int(rng.integers(1, 200))
        s0 = int(rng.integers(0, 40000 - n))
        buf = dev(np.concatenate([np.zeros(16, np.uint8), full[s0 * SECTOR:(s0 + n) * SECTOR]]))
        keep.append(buf)
        images.append((buf.data_ptr() + 16, n * SECTOR))
        wants.append(want(s0, n))
    order = rng.permutation(len(images))
    images = [images[i] for i in order]
    wants = [wants[i] for i in order]
    assert sum(w.size for w in wants) > 500
    with cv.master_build(files) as m:
        for cfg in range(1, len(cv.kernel_configs()) + 1):
            with cv.scan(m, images, kernel_config=cfg) as r:
                for k in range(len(images)):
                    assert_same(r.matches(k), wants[k], f"configuration {cfg}, image {k}")


def _batch_images(n_images, seed):
    """Images of uneven sizes carved out of one device buffer, plus their oracle results."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(0, 4000, size=n_images)
    sizes[3] = 0
    sizes[5] = 1
    plan = synth.config_plan(f"small:{int(sizes.sum()) + 64}:60:{seed}")
    full = plan.image_host()
    files = plan.masters_host()
    whole = dev(full)
    images, wants, a = [], [], 0
    for n in sizes.tolist():
        images.append((whole.data_ptr() + a * SECTOR, n * SECTOR))
        wants.append(oracle.match_hash(full[a * SECTOR:(a + n) * SECTOR], files))
        a += n
    return files, whole, images, wants


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_graph_equals_oracle_per_image(cv, autotune, tmp_path):
    files, whole, images, wants = _batch_images(40, 31)
    with cv.master_build(files) as m:
        cache = str(tmp_path / "tune.txt") if autotune else None
        with cv.batch_create(m, images, autotune=autotune, tune_cache=cache) as b:
            info = b.info()
            assert info["tensor_maps"] == 1 and info["segments"] == sum(1 for w in images if w[1] >= SECTOR)
            for run in range(2):  # replays give the same result
                b.run()
                total = b.wait()
                assert total == sum(w.size for w in wants)
                for k in range(len(images)):
                    assert_same(cv.device_matches_to_numpy(b.matches(k)), wants[k], f"run {run} image {k}")
                # the scan launch inside the graph is timed on every replay
                assert b.info()["scan_ms"] > 0, run
        if autotune:
            assert open(cache).read().strip()
            with cv.batch_create(m, images, autotune=True, tune_cache=cache) as b2:
                assert b2.info()["tuned"] == 0  # served from the cache


@pytest.mark.parametrize("sig", [0, 2])
@pytest.mark.parametrize("sorted_copy", [False, True])
@pytest.mark.parametrize("bloom_mode", ["off", "on"])
def test_batch_table_variants_equal_oracle(cv, sig, sorted_copy, bloom_mode):
    """Every table variant the batch tuner can choose, forced one at a time on a hash-layout
    master without a Bloom filter: the master's own table or its sorted copy, probed directly or
    through a filter the batch builds. Each must give the oracle's result per image."""
    files, whole, images, wants = _batch_images(30, 41 + sig)
    bloom = cv.CV_BATCH_BLOOM_ON if bloom_mode == "on" else cv.CV_BATCH_BLOOM_OFF
    with cv.master_build(files, signature=sig, bloom_bits_per_key=0, max_load=0.9) as m:
        assert m.info()["bloom_bytes"] == 0 and m.info()["layout"] == cv.CV_LAYOUT_HASH
        with cv.batch_create(m, images, bloom=bloom, sorted_copy=sorted_copy) as b:
            info = b.info()
            assert info["layout"] == (cv.CV_LAYOUT_SORTED if sorted_copy else cv.CV_LAYOUT_HASH)
            assert info["bloom"] == (1 if bloom_mode == "on" else 0)
            for run in range(2):
                b.run()
                assert b.wait() == sum(w.size for w in wants)
                for k in range(len(images)):
                    assert_same(cv.device_matches_to_numpy(b.matches(k)), wants[k], f"run {run} image {k}")


@pytest.mark.parametrize("layout", [0, 1])
def test_batch_tuner_reports_its_choice(cv, layout, tmp_path):
    """The tuner searches configuration x layout x Bloom on the batch and reports what it chose;
    whatever it chose, the results are the oracle's, and a second batch takes the choice from the
    cache file."""
    files, whole, images, wants = _batch_images(30, 45)
    cache = str(tmp_path / "tune.txt")
    with cv.master_build(files, bloom_bits_per_key=0, max_load=0.9, layout=layout) as m:
        with cv.batch_create(m, images, autotune=True, tune_cache=cache) as b:
            info = b.info()
            assert info["tuned"] == 1
            assert info["layout"] in (cv.CV_LAYOUT_HASH, cv.CV_LAYOUT_SORTED)
            if layout == cv.CV_LAYOUT_SORTED:
                assert info["layout"] == cv.CV_LAYOUT_SORTED  # a sorted master has no hash copy
            b.run()
            assert b.wait() == sum(w.size for w in wants)
            for k in range(len(images)):
                assert_same(cv.device_matches_to_numpy(b.matches(k)), wants[k], f"image {k}")
        line = open(cache).read().split()
        assert len(line) == 4 and line[1] == info["config_name"]
        assert int(line[3]) == info["layout"] and int(line[2]) == info["bloom"]
        with cv.batch_create(m, images, autotune=True, tune_cache=cache) as b2:
            i2 = b2.info()
            assert i2["tuned"] == 0
            assert (i2["kernel_config"], i2["layout"], i2["bloom"]) == (info["kernel_config"], info["layout"],
                                                                        info["bloom"])
            b2.run()
            b2.wait()
            for k in range(len(images)):
                assert_same(cv.device_matches_to_numpy(b2.matches(k)), wants[k], f"cached, image {k}")


@pytest.mark.parametrize("cfg", range(9))
def test_every_kernel_config_serves_every_table_kind(cv, cfg):
    """Each kernel configuration is built for all four signatures and both layouts: scans with it
    give the oracle's result for a 64-bit signature and the sorted layout alike."""
    assert len(cv.kernel_configs()) == 9
    files, whole, images, wants = _batch_images(6, 47)
    img, want = images[0], wants[0]
    for sig, layout in ((3, cv.CV_LAYOUT_SORTED), (1, cv.CV_LAYOUT_HASH)):
        with cv.master_build(files, signature=sig, layout=layout) as m:
            with cv.scan(m, [img], kernel_config=cfg + 1) as r:
                assert_same(r.matches(0), want, f"config {cfg} sig {sig}")


def test_scan_reports_configuration_and_signature_defaults(cv):
    """cv_scan_stats.kernel_config names the configuration a scan used: by default configuration
    0 for MD5 and MD5 without padding, the 128-byte-stage one for djb2-64 and CRC64 (their scans
    are bound by staging), or the one the caller selects; the result is the same in every case."""
    files, whole, images, wants = _batch_images(6, 49)
    names = cv.kernel_configs()
    light = names.index("t128_x1_s2_b128_p2")
    for sig, expect in ((0, 0), (1, 0), (2, light), (3, light)):
        with cv.master_build(files, signature=sig) as m:
            with cv.scan(m, [images[1]]) as r:
                assert r.stats()["kernel_config"] == expect
                assert_same(r.matches(0), wants[1], f"sig {sig}")
            with cv.scan(m, [images[1]], kernel_config=3) as r:
                assert r.stats()["kernel_config"] == 2
                assert_same(r.matches(0), wants[1], f"sig {sig} config 2")
    frag_files = [f[: f.size // 64 * 64] for f in files]
    with cv.master_build(frag_files, unit=cv.CV_UNIT_FRAGMENT) as m, cv.scan(m, [images[1]]) as r:
        assert r.stats()["kernel_config"] == -1


def test_scan_output_room_follows_previous_scans(cv):
    """A scan launches its expand pass with room sized from the previous scan against the same
    table: scans whose match counts rise (room too small: the pass reruns into an exact buffer)
    and fall (room to spare), an image with no sectors, host and device results, all equal the
    oracle's."""
    big = synth.config_plan("small:60000:200:53")
    small = synth.make_plan(54, 5000, big.file_nsect, 0.1, master_seed=big.master_seed)
    files = big.masters_host()
    imgs = {"big": big.image_host(), "small": small.image_host(), "empty": np.zeros(100, np.uint8)}
    wants = {k: oracle.match_hash(v, files) for k, v in imgs.items()}
    assert wants["big"].size > 1.25 * wants["small"].size + 1024 and wants["small"].size > 0
    devs = {k: dev(v) for k, v in imgs.items()}
    with cv.master_build(files) as m:
        for step, k in enumerate(["small", "big", "big", "small", "empty", "big", "small"]):
            with cv.scan(m, [devs[k]]) as r:
                assert_same(r.matches(0), wants[k], f"step {step} {k}")
            with cv.scan(m, [devs[k]], keep_on_device=True) as r:
                assert r.count(0) == wants[k].size
                if wants[k].size:
                    assert_same(cv.device_matches_to_numpy(r.matches(0)), wants[k], f"step {step} {k}, on device")


def test_batch_capacity_overflow_reported(cv):
    files, whole, images, wants = _batch_images(12, 33)
    total = sum(w.size for w in wants)
    assert total > 10
    with cv.master_build(files) as m, cv.batch_create(m, images, match_capacity=10) as b:
        b.run()
        with pytest.raises(cv.CVError) as e:
            b.wait()
        assert e.value.code == cv.CV_ERANGE


def test_server_results_equal_solo_scans(cv):
    """Requests of mixed sizes arriving together: each result equals the oracle and the solo
    scan of the same image, while work units of many requests share launches."""
    plan = synth.config_plan("small:120000:80:51")
    files = plan.masters_host()
    full = plan.image_host()
    rng = np.random.default_rng(9)
    cuts = []
    for k in range(30):
        n = int(rng.integers(1, 40)) if k % 5 else int(rng.integers(3000, 20000))
        a = int(rng.integers(0, 120000 - n))
        cuts.append((a, n))
    cuts.append((0, 0))
    pinned = torch.from_numpy(full).pin_memory()
    with cv.master_build(files) as m:
        # work units of 1 MiB and a 6 MiB budget force units of big requests to take turns
        with cv.server_create(m, work_unit_bytes=1 << 20, hbm_budget_bytes=6 << 20, max_live=8) as srv:
            tickets = []
            for k, (a, n) in enumerate(cuts):
                img = pinned[a * SECTOR:(a + n) * SECTOR] if k % 2 else np.ascontiguousarray(
                    full[a * SECTOR:(a + n) * SECTOR])
                tickets.append(srv.submit(img, tag=k))
            dimg = dev(full[5000 * SECTOR:9000 * SECTOR])
            tdev = srv.submit(dimg, tag=99)
            for k, t in enumerate(tickets):
                r = srv.poll(t, timeout_ms=60000)
                assert r is not None
                a, n = cuts[k]
                want = oracle.match_hash(full[a * SECTOR:(a + n) * SECTOR], files)
                assert_same(r.matches(0), want, f"request {k}")
                r.close()
            r = srv.poll(tdev, timeout_ms=60000)
            assert_same(r.matches(0), oracle.match_hash(full[5000 * SECTOR:9000 * SECTOR], files), "device request")
            r.close()
            st = srv.stats()
            assert st["completed"] == len(cuts) + 1 and st["failed"] == 0
            assert st["peak_bytes_in_flight"] <= 6 << 20
            assert st["p99_ms"] >= st["p50_ms"] > 0
        # the solo scan of one of the big requests gives the same list
        a, n = cuts[0]
        with cv.scan(m, [np.ascontiguousarray(full[a * SECTOR:(a + n) * SECTOR])]) as r:
            assert_same(r.matches(0), oracle.match_hash(full[a * SECTOR:(a + n) * SECTOR], files), "solo")


@pytest.mark.parametrize("cap", [1, 3 << 20, 2**64 - 1])
def test_server_copy_cap(cv, cap):
    """However many copy bytes may be queued at once (one unit, a few, no limit), every request,
    large and small, submitted together, gets the oracle's matches."""
    plan = synth.config_plan("small:60000:60:52")
    files = plan.masters_host()
    full = plan.image_host()
    pinned = torch.from_numpy(full).pin_memory()
    cuts = [(0, 60000), (100, 7), (30000, 25000), (5, 1), (59000, 1000), (7000, 33)]
    with cv.master_build(files) as m:
        with cv.server_create(m, work_unit_bytes=1 << 20, copy_streams=3, max_copy_bytes=cap) as srv:
            tickets = [srv.submit(pinned[a * SECTOR:(a + n) * SECTOR], tag=k) for k, (a, n) in enumerate(cuts)]
            for k, t in enumerate(tickets):
                r = srv.poll(t, timeout_ms=60000)
                a, n = cuts[k]
                assert_same(r.matches(0), oracle.match_hash(full[a * SECTOR:(a + n) * SECTOR], files), f"request {k}")
                r.close()


def test_server_opts_without_copy_cap_field(cv):
    """Options of the size before max_copy_bytes existed are accepted (the cap takes its
    default); anything shorter is refused."""
    files = [synth.random_sectors(4, 64)]
    lib = cv.load()
    with cv.master_build(files) as m:
        for size, ok in [(ctypes.sizeof(cv.cv_server_opts) - 8, True), (ctypes.sizeof(cv.cv_server_opts) - 12, False)]:
            o = cv.cv_server_opts(size, 0, 0, 0, 0, 0, 123)
            h = ctypes.c_void_p()
            rc = lib.cv_server_create(m.handle, ctypes.byref(o), ctypes.byref(h))
            assert (rc == cv.CV_OK) == ok, (size, rc)
            if h.value:
                srv = cv.Server(h.value)
                t = srv.submit(np.ascontiguousarray(files[0]))
                r = srv.poll(t, timeout_ms=60000)
                assert r.count(0) == 64
                r.close()
                srv.close()


def test_server_poll_nonblocking_and_unknown_ticket(cv):
    files = [synth.random_sectors(3, 64)]
    with cv.master_build(files) as m, cv.server_create(m) as srv:
        with pytest.raises(cv.CVError):
            srv.poll(12345, timeout_ms=0)
        t = srv.submit(np.ascontiguousarray(files[0]))
        r = None
        for _ in range(2000):
            r = srv.poll(t, timeout_ms=10)
            if r is not None:
                break
        assert r is not None and r.count(0) == 64
        r.close()


def test_concurrent_scans_on_separate_streams(cv):
    """Separate scans may run at the same time from several host threads, each on its own
    stream (the library's shared state is the device context and its memory pool)."""
    import threading

    plan = synth.config_plan("small:20000:30:77")
    files = plan.masters_host()
    img = plan.image_host()
    want = oracle.match_hash(img, files)
    with cv.master_build(files) as m:
        dev = torch.from_numpy(img).cuda()
        errors, results = [], {}

        def worker(k):
            try:
                s = torch.cuda.Stream()
                got = []
                for rep in range(5):
                    src = dev if (k + rep) % 2 == 0 else img  # device and host images alike
                    with cv.scan(m, [src], stream=s.cuda_stream, chunk_bytes=(3 + k) * 4096) as r:
                        got.append(r.matches(0))
                results[k] = got
            except Exception as e:  # reported below
                errors.append(e)

        def fresh_thread_noalloc():
            try:
                out = torch.empty(16 * (want.size + 8), dtype=torch.uint8, device="cuda")
                rc, n = cv.scan_noalloc(m, dev, out, want.size + 8)
                results["noalloc"] = np.frombuffer(out[: n * 16].cpu().numpy().tobytes(), cv.MATCH_DTYPE)
            except Exception as e:
                errors.append(e)

        threads = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        threads.append(threading.Thread(target=fresh_thread_noalloc))
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for k in range(4):
            for got in results[k]:
                assert np.array_equal(got, want)
        assert np.array_equal(results["noalloc"], want)


def test_permuted_master_order_only_relabels(cv):
    """Metamorphic: permuting the master files permutes file_ids and nothing else; the scan also
    reports how many disk sectors matched (host and device images alike)."""
    plan = synth.config_plan("small:30000:40:91")
    img = plan.image_host()
    files = plan.masters_host()
    perm = np.random.default_rng(5).permutation(len(files))
    dev = torch.from_numpy(img).cuda()
    with cv.master_build(files) as m, cv.scan(m, [dev, img], chunk_bytes=777 * 512) as r:
        base = r.matches(0)
        assert np.array_equal(r.matches(1), base)
        assert r.stats()["hit_sectors"] == 2 * np.unique(base["disk_sector"]).size
    with cv.master_build([files[k] for k in perm]) as m, cv.scan(m, [dev]) as r:
        got = r.matches(0)
    relabelled = got.copy()
    relabelled["file_id"] = perm[got["file_id"]]
    relabelled.sort(order=["disk_sector", "file_id", "file_sector"])
    assert np.array_equal(relabelled, base)
