"""Seeded fuzzing of the GPU path against the oracle: each case draws an image and master files
from a few reusable sector or fragment shapes (so matches, duplicates, fills and ragged tails are
common) and random options (signature, layout, position keying, Bloom filter, load cap, unit,
host or device image, streaming chunk size), then compares the scan with the oracle exactly."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR, FRAG = 512, 64


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def draw(rng, unit, n_pieces):
    base = rng.integers(0, 256, 6 * unit, dtype=np.uint8)
    shapes = [base[k * unit:(k + 1) * unit] for k in range(6)]
    shapes += [np.zeros(unit, np.uint8), np.full(unit, 0x41, np.uint8)]
    near = np.zeros(unit, np.uint8)
    near[-1] = 1
    shapes.append(near)

    def blob(n):
        parts = []
        for _ in range(n):
            r = rng.random()
            if r < 0.75:
                parts.append(shapes[int(rng.integers(0, len(shapes)))])
            elif r < 0.9:
                parts.append(rng.integers(0, 256, unit, dtype=np.uint8))
            else:
                parts.append(rng.integers(0, 256, int(rng.integers(1, unit)), dtype=np.uint8))
        return np.concatenate(parts) if parts else np.zeros(0, np.uint8)

    image = blob(n_pieces)
    files = [blob(int(rng.integers(0, 12))) for _ in range(int(rng.integers(1, 6)))]
    return image, files


@pytest.mark.parametrize("seed", range(200))
def test_fuzz_against_oracle(cv, seed):
    rng = np.random.default_rng(1000 + seed)
    frag = seed % 4 == 3
    if frag:
        image, files = draw(rng, FRAG, int(rng.integers(0, 300 if seed % 5 else 20000)))
        # windows at 4-byte offsets: shift the image by 0-3 words
        image = np.concatenate([rng.integers(0, 256, 4 * int(rng.integers(0, 4)), dtype=np.uint8), image])
        sig = int(rng.choice([0, 1, 2]))
        kw = dict(unit=cv.CV_UNIT_FRAGMENT, signature=sig)
        want = oracle.frag_match(image, files)
        base = 0
    else:
        # most images fit in one scan tile (256 sectors); every fifth spans many
        image, files = draw(rng, SECTOR, int(rng.integers(0, 200 if seed % 5 else 3000)))
        sig = int(rng.integers(0, 4))
        position = bool(rng.random() < 0.3)
        base = int(rng.integers(0, 16)) if position else 0
        kw = dict(signature=sig, position_mode=1 if position else 0)
        want = oracle.match_position(image, files, base) if position else oracle.match_hash(image, files)
    kw.update(layout=int(rng.integers(0, 3)), bloom_bits_per_key=int(rng.choice([0, 8, 16])),
              max_load=float(rng.choice([0.25, 0.5, 0.9])))
    on_device = bool(rng.random() < 0.5)
    chunk = int(rng.integers(1, 64)) * SECTOR
    with cv.master_build(files, **kw) as m:
        src = torch.from_numpy(image).cuda() if (on_device and image.size) else image
        with cv.scan(m, [src], chunk_bytes=chunk, base_offset=base) as r:
            got = r.matches(0)
    assert np.array_equal(got, want), (seed, kw, on_device, chunk)
    if frag or seed % 3 or image.size < SECTOR:
        return
    # the same case through the batched, served and allocation-free entry points (sector tables,
    # clusters counted from each image's sector 0)
    if kw.get("position_mode"):
        want = oracle.match_position(image, files, 0)
    d = torch.from_numpy(image).cuda()
    with cv.master_build(files, **kw) as m:
        with cv.batch_create(m, [d, (d.data_ptr(), (image.size // 2) // SECTOR * SECTOR)],
                             autotune=bool(seed % 2)) as b:
            b.run()
            b.wait()
            assert np.array_equal(cv.device_matches_to_numpy(b.matches(0)), want)
            half = image[: (image.size // 2) // SECTOR * SECTOR]
            want_half = oracle.match_position(half, files, 0) if kw.get("position_mode") else oracle.match_hash(half, files)
            assert np.array_equal(cv.device_matches_to_numpy(b.matches(1)), want_half)
        with cv.server_create(m, work_unit_bytes=int(rng.integers(1, 9)) * SECTOR, hbm_budget_bytes=1 << 20) as srv:
            t = srv.submit(np.ascontiguousarray(image))
            r = srv.poll(t, timeout_ms=60000)
            assert np.array_equal(r.matches(0), want)
            r.close()
        out = torch.empty(16 * (want.size + 4), dtype=torch.uint8, device="cuda")
        rc, n = cv.scan_noalloc(m, d, out, want.size + 4)
        assert rc == cv.CV_OK and np.array_equal(np.frombuffer(out[: n * 16].cpu().numpy().tobytes(), cv.MATCH_DTYPE), want)
