"""Master builds from many files in every kind of memory: the copy stage merges contiguous
files, gathers those in this GPU's memory with one kernel (4 MiB pieces, 16-byte or byte
copies), stages short host runs through pinned memory and leaves long ones to the driver. The
tables must be the oracle's whatever the mix: the scans' matches are compared bit for bit."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def mixed_files(rng, n, unit, max_units, big_every=0):
    """n files of 1..max_units units (some with a ragged tail), as numpy arrays."""
    out = []
    for k in range(n):
        units = int(rng.integers(1, max_units + 1))
        if big_every and k % big_every == 0:
            units = (6 << 20) // unit  # longer than one gather piece and than the host staging cut
        tail = int(rng.integers(1, unit)) if k % 5 == 0 else 0
        out.append(rng.integers(0, 256, units * unit + tail, dtype=np.uint8))
    return out


def kind_of(k):
    return (k // 10) % 5  # blocks of ten consecutive files share a kind


def place(files, keep):
    """The files in memory of five kinds, in blocks of ten consecutive files; returns the
    cv_buf-like objects."""
    packed = [f for k, f in enumerate(files) if kind_of(k) == 0]
    dev_packed = torch.from_numpy(np.concatenate(packed)).cuda()  # back to back: merged runs
    gap = 48
    scattered_len = sum(f.size + gap for k, f in enumerate(files) if kind_of(k) == 1) + 64
    dev_gapped = torch.zeros(scattered_len, dtype=torch.uint8, device="cuda")
    objs = [None] * len(files)
    off_packed = 0
    off_gapped = 0
    for k, f in enumerate(files):
        kind = kind_of(k)
        if kind == 0:
            objs[k] = dev_packed[off_packed:off_packed + f.size]
            off_packed += f.size
        elif kind == 1:  # one device buffer, files apart
            dev_gapped[off_gapped:off_gapped + f.size] = torch.from_numpy(f).cuda()
            objs[k] = dev_gapped[off_gapped:off_gapped + f.size]
            off_gapped += f.size + gap
        elif kind == 2:  # pageable host
            objs[k] = np.ascontiguousarray(f)
        elif kind == 3:  # pinned host
            objs[k] = torch.from_numpy(f).pin_memory()
        else:  # its own device allocation, starting 3 bytes in (misaligned source)
            t = torch.zeros(f.size + 3, dtype=torch.uint8, device="cuda")
            t[3:] = torch.from_numpy(f).cuda()
            objs[k] = (t.data_ptr() + 3, f.size)
            keep.append(t)
    keep += [dev_packed, dev_gapped]
    return objs


def image_with_plants(rng, files, unit, n_units, n_plants):
    img = rng.integers(0, 256, n_units * unit, dtype=np.uint8)
    for _ in range(n_plants):
        f = files[int(rng.integers(0, len(files)))]
        whole = f.size // unit
        u = int(rng.integers(0, whole))
        at = int(rng.integers(0, n_units))
        img[at * unit:(at + 1) * unit] = f[u * unit:(u + 1) * unit]
    return img


@pytest.mark.parametrize("seed", [31, 32])
def test_sector_tables_from_many_files_in_mixed_memory(cv, seed):
    rng = np.random.default_rng(seed)
    files = mixed_files(rng, 2500, SECTOR, 4, big_every=710)  # big ones: device, device, pageable, pinned
    keep = []
    objs = place(files, keep)
    img = image_with_plants(rng, files, SECTOR, 40000, 3000)
    want = oracle.match_hash(img, files)
    assert want.size > 2000
    with cv.master_build(objs) as m:
        assert m.info()["n_sectors"] == sum(f.size // SECTOR for f in files)
        with cv.scan(m, [torch.from_numpy(img).cuda()]) as r:
            assert np.array_equal(r.matches(0), want)


def test_fragment_tables_from_many_files_in_mixed_memory(cv):
    rng = np.random.default_rng(33)
    files = mixed_files(rng, 1500, 64, 20)
    keep = []
    objs = place(files, keep)
    img = image_with_plants(rng, files, 64, 30000, 2000)
    want = oracle.frag_match(img, files)
    assert want.size > 1000
    with cv.master_build(objs, unit=1, signature=2) as m:
        with cv.scan(m, [torch.from_numpy(img).cuda()]) as r:
            assert np.array_equal(r.matches(0), want)


def test_empty_and_tail_only_files_between_others(cv):
    rng = np.random.default_rng(34)
    a = rng.integers(0, 256, 8 * SECTOR, dtype=np.uint8)
    b = rng.integers(0, 256, 3 * SECTOR, dtype=np.uint8)
    dev = torch.from_numpy(np.concatenate([a, b])).cuda()
    tail = torch.from_numpy(rng.integers(0, 256, 100, dtype=np.uint8)).cuda()
    objs = [dev[:a.size], (0, 0), tail, np.zeros(0, np.uint8), dev[a.size:]]
    files = [a, np.zeros(0, np.uint8), tail.cpu().numpy(), np.zeros(0, np.uint8), b]
    img = np.concatenate([b, a, rng.integers(0, 256, 5 * SECTOR, dtype=np.uint8)])
    with cv.master_build(objs) as m:
        assert m.info()["n_sectors"] == 11
        with cv.scan(m, [torch.from_numpy(img).cuda()]) as r:
            assert np.array_equal(r.matches(0), oracle.match_hash(img, files))
