"""The GPU's signature arithmetic, value by value, against the oracle.

Match lists alone cannot catch a wrong 64-bit signature: equal bytes hash equally whatever the
function, and byte confirmation drops every false candidate, so a consistent error leaves every
list unchanged. These tests read the signatures themselves out of the kernels that compute them
in scans and table builds (cv_sector_signatures: the scan kernel's per-sector code; and
cv_window_signatures: the fragment kernels' per-window code, the rolled djb2 included) and
compare each one with the oracle: MD5 (RFC 1321), MD5 without the padding block (Section 2.1),
djb2-64 (Eq. 1) and CRC64 with generator x^64 + x^4 + x^3 + x + 1 (Section 2.1)."""
import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512
SIG_BYTES = {0: 16, 1: 16, 2: 8, 3: 8}  # bytes of the 16-byte output that hold the signature


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


@pytest.fixture(scope="module")
def sector_image():
    """About a million sectors of every class the generator makes (random, all-zero, text,
    planted master sectors), with edge cases in front: one-byte fills, single set bits at both
    ends of the sector (the CRC's highest and lowest message coefficients), an all-ones sector,
    and a ragged count (not a multiple of any tile)."""
    n = (1 << 20) - 5
    plan = synth.config_plan(f"small:{n}:300:91")
    img = plan.image_host().reshape(-1, SECTOR).copy()
    img[0] = 0
    img[1] = 0xFF
    img[2] = 0
    img[2, 0] = 0x80  # the first message bit
    img[3] = 0
    img[3, SECTOR - 1] = 0x01  # the last message bit
    img[4] = 0x5A
    rng = np.random.default_rng(92)
    for k in range(5, 40):
        img[k] = 0
        img[k, int(rng.integers(0, SECTOR))] = 1 << int(rng.integers(0, 8))
    return img.reshape(-1)


@pytest.mark.parametrize("sig", [0, 1, 2, 3])
def test_sector_signatures_equal_oracle(cv, sector_image, sig):
    n = sector_image.size // SECTOR
    d = torch.from_numpy(sector_image).cuda()
    out = torch.zeros(n * 16, dtype=torch.uint8, device="cuda")
    triv = torch.zeros(n, dtype=torch.uint8, device="cuda")
    cv.sector_signatures(d.data_ptr(), n, sig, out.data_ptr(), triv.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(n, 16)
    want = oracle.signatures(sector_image, sig)
    k = SIG_BYTES[sig]
    bad = np.nonzero((got[:, :k] != want[:, :k]).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} of {n} sectors differ, first {bad[:5]}"
    # the exclusion flags, for a sample, against the oracle's rule
    t = triv.cpu().numpy()
    for i in list(range(40)) + list(range(1000, n, 9973)):
        assert t[i] == int(oracle.sector_trivial(sector_image[i * SECTOR:(i + 1) * SECTOR]))


def test_sector_digests_is_md5_signature(cv, sector_image):
    n = 4096
    d = torch.from_numpy(sector_image[: n * SECTOR]).cuda()
    a = torch.zeros(n * 16, dtype=torch.uint8, device="cuda")
    b = torch.zeros(n * 16, dtype=torch.uint8, device="cuda")
    cv.sector_digests(d.data_ptr(), n, a.data_ptr())
    cv.sector_signatures(d.data_ptr(), n, cv.CV_SIG_MD5, b.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert np.array_equal(a.cpu().numpy().reshape(n, 16), oracle.md5_sectors(sector_image[: n * SECTOR]))


def test_signature_arguments_are_checked(cv):
    d = torch.zeros(4 * SECTOR, dtype=torch.uint8, device="cuda")
    out = torch.zeros(4 * 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(cv.CVError):
        cv.sector_signatures(d.data_ptr(), 4, 4, out.data_ptr())
    with pytest.raises(cv.CVError):
        cv.sector_signatures(d.data_ptr() + 4, 3, 2, out.data_ptr())
    with pytest.raises(cv.CVError):
        cv.window_signatures(d.data_ptr(), 4 * SECTOR, cv.CV_SIG_CRC64, out.data_ptr())


@pytest.mark.parametrize("sig", [0, 1, 2])
@pytest.mark.parametrize("n_bytes", [64, 64 + 4 * 543 + 3, (3 << 20) + 37])
def test_window_signatures_equal_oracle(cv, sig, n_bytes):
    """Every window of a ragged image: the rolled djb2 crosses lane and tile boundaries (each lane
    computes its first window directly and rolls the rest; a tile is 544 windows), and the last
    window ends short of the image's end when n_bytes is not a multiple of 4."""
    rng = np.random.default_rng(93 + sig)
    img = rng.integers(0, 256, n_bytes, dtype=np.uint8)
    img[1000:1300] = 0  # zero windows
    img[5000:5100] = 0xFF
    buf = torch.zeros((n_bytes + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
    buf[:n_bytes] = torch.from_numpy(img).cuda()
    n_win = (n_bytes - 64) // 4 + 1
    out = torch.zeros(n_win * 16, dtype=torch.uint8, device="cuda")
    cv.window_signatures(buf.data_ptr(), n_bytes, sig, out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(n_win, 16)
    want = oracle.window_signatures(img, sig)
    k = SIG_BYTES[sig]
    bad = np.nonzero((got[:, :k] != want[:, :k]).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} of {n_win} windows differ, first {bad[:5]}"


def test_window_signatures_of_fragment_workload(cv):
    """The fragment workload's image (logos planted at 4-byte offsets in the usual sector mix),
    every window under the rolled djb2."""
    fp = synth.make_frag_plan(94, 4 << 20, 60)
    img = fp.image_host()
    d = torch.from_numpy(img).cuda()
    n_win = (img.size - 64) // 4 + 1
    out = torch.zeros(n_win * 16, dtype=torch.uint8, device="cuda")
    cv.window_signatures(d.data_ptr(), img.size, cv.CV_SIG_DJB2_64, out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(n_win, 16)[:, :8]
    assert np.array_equal(got, oracle.window_signatures(img, 2)[:, :8])
