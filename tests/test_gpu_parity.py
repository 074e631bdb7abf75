"""GPU parity: the CUDA path through the C ABI against the CPU oracle, on the same seeded inputs.

Everything here is integer work, so the bar is bit-exact: identical digests, identical trivial
flags, identical sorted match lists.
"""
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
