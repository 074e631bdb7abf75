"""cv_carve, the C command-line tool written against include/cv.h alone, on real files: its
printed matches equal the oracle's for sectors, position-keyed tables, djb2 and fragments."""
import subprocess

import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def exe(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import build

    return build.build_cli()


def run(exe, args):
    r = subprocess.run([exe, *args], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    rows = [tuple(int(x) for x in line.split()) for line in r.stdout.splitlines()]
    return rows


def as_rows(image_index, arr):
    return [(image_index, int(a), int(b), int(c)) for a, b, c in zip(arr["disk_sector"], arr["file_id"], arr["file_sector"])]


def write(tmp_path, name, arr):
    p = tmp_path / name
    p.write_bytes(np.ascontiguousarray(arr).tobytes())
    return str(p)


def test_cli_sectors_positions_signatures(exe, tmp_path):
    plan = synth.config_plan("small:12000:20:41")
    img = plan.image_host()
    files = plan.masters_host()
    # a second image that is a ragged slice of the first
    img2 = img[7 * 512 + 100: 9000 * 512 + 77]
    paths = [write(tmp_path, f"m{f}", x) for f, x in enumerate(files)]
    i1, i2 = write(tmp_path, "img1", img), write(tmp_path, "img2", img2)
    want = as_rows(0, oracle.match_hash(img, files)) + as_rows(1, oracle.match_hash(img2, files))
    assert run(exe, [i1, i2, "--", *paths]) == want
    assert run(exe, ["-s", "2", i1, i2, "--", *paths]) == want
    want_p = as_rows(0, oracle.match_position(img, files, 5)) + as_rows(1, oracle.match_position(img2, files, 5))
    assert run(exe, ["-p", "5", i1, i2, "--", *paths]) == want_p


def test_cli_fragments(exe, tmp_path):
    fp = synth.make_frag_plan(44, (2 << 20) + 3, 40, header_frac=0.3)
    img = fp.image_host()
    logos = fp.logos()
    paths = [write(tmp_path, f"l{f}", x) for f, x in enumerate(logos)]
    want = as_rows(0, oracle.frag_match(img, logos))
    assert len(want) > 100
    assert run(exe, ["-f", write(tmp_path, "img", img), "--", *paths]) == want
