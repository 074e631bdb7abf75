"""The C ABI library builds, loads and exports every function include/cv.h declares (no GPU).

On a machine without a usable GPU the library must refuse work (CV_ENODEV): it has no CPU path.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "cv.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(cv_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0901_1307_gb300 import build, cv

    build.build()
    return cv.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cv_master_build", "cv_scan", "cv_matches", "cv_free"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_0901_1307_gb300 import cv

    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(cv.EXPORTS) <= set(declared_functions())


def test_strerror_and_null_arguments(lib):
    from paper_0901_1307_gb300 import cv

    assert cv.strerror(cv.CV_OK) == "ok"
    assert cv.strerror(cv.CV_ENODEV) == "no usable CUDA device"
    out = ctypes.c_void_p()
    assert lib.cv_master_build(None, 1, None, ctypes.byref(out)) == cv.CV_EINVAL
    assert lib.cv_scan(None, None, 0, None, ctypes.byref(out)) == cv.CV_EINVAL
    assert lib.cv_matches(None, 0, None, None) == cv.CV_EINVAL
    st = cv.cv_probe_stats()
    st.struct_size = ctypes.sizeof(st)
    assert lib.cv_probe_profile(None, None, 0, 0, ctypes.byref(st), None) == cv.CV_EINVAL
    assert lib.cv_probe_profile(None, None, 0, 0, None, None) == cv.CV_EINVAL
    lib.cv_free(None)


def test_no_cpu_path_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_0901_1307_gb300 import cv

    with pytest.raises(cv.CVError) as e:
        cv.master_build([bytes(1024)])
    assert e.value.code == cv.CV_ENODEV


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets the C compiler gives
    the header's struct (a field added to one side only shows up here)."""
    from paper_0901_1307_gb300 import cv

    structs = [n for n in dir(cv) if n.startswith("cv_") and isinstance(getattr(cv, n), type)
               and issubclass(getattr(cv, n), ctypes.Structure)]
    assert {"cv_master_opts", "cv_scan_opts", "cv_master_info", "cv_batch_opts", "cv_server_opts"} <= set(structs)
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cv.h"', "int main(void) {"]
    for n in structs:
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in getattr(cv, n)._fields_:
            lines.append(f'  printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess

    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.splitlines())
    for n in structs:
        st = getattr(cv, n)
        assert int(got[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(st, f).offset, f"{n}.{f}"


def test_master_options_checked_before_the_device(lib):
    """Option validation is host logic: without a GPU a well-formed request gets CV_ENODEV and a
    malformed one CV_EINVAL (struct too small, unknown position mode or signature)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_0901_1307_gb300 import cv

    h = ctypes.c_void_p()

    def build(size, position_mode=0, signature=0):
        o = cv.cv_master_opts(size, 0.0, 0, signature, None, position_mode, 0)
        return lib.cv_master_build(None, 0, ctypes.byref(o), ctypes.byref(h))

    full = ctypes.sizeof(cv.cv_master_opts)
    assert build(full) == cv.CV_ENODEV
    assert build(full, position_mode=cv.CV_POSITION_CLUSTER) == cv.CV_ENODEV
    assert build(24) == cv.CV_ENODEV                   # the size before position_mode existed
    assert build(24, position_mode=7) == cv.CV_ENODEV  # not read at that size
    assert build(20) == cv.CV_EINVAL
    assert build(full, position_mode=2) == cv.CV_EINVAL
    assert build(full, signature=4) == cv.CV_EINVAL


def test_cli_builds_and_refuses_without_gpu(lib, tmp_path):
    """cv_carve, the C command-line tool, links against libcv.so through include/cv.h alone;
    without a GPU it reports the library's error (exit 2); a bad command line exits 1."""
    torch = pytest.importorskip("torch")
    import subprocess

    from paper_0901_1307_gb300 import build

    exe = build.build_cli()
    img = tmp_path / "img"
    img.write_bytes(bytes(4096))
    r = subprocess.run([exe, str(img)], capture_output=True, text=True)
    assert r.returncode == 1 and "usage" in r.stderr
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([exe, str(img), "--", str(img)], capture_output=True, text=True)
    assert r.returncode == 2 and "no usable CUDA device" in r.stderr


def test_buffer_lists_marshal_to_cv_buf_arrays():
    """The binding's three ways of passing buffer lists give the same cv_buf array: elements one
    by one, (pointer, bytes) tuples converted at once, and an (n, 2) uint64 descriptor array."""
    import ctypes

    import numpy as np

    from paper_0901_1307_gb300 import cv

    a = np.arange(3000, dtype=np.uint8)
    b = np.zeros(0, np.uint8)
    rows = [(a.ctypes.data, a.nbytes), (0, 0), (a.ctypes.data + 512, 1024)]

    def as_pairs(arr, n):
        return [(arr[i].data or 0, arr[i].n_bytes) for i in range(n)]

    one_by_one, keep1 = cv._bufs([a, b, (a.ctypes.data + 512, 1024)])
    tuples, keep2 = cv._bufs(rows)
    desc, keep3 = cv._bufs(np.array(rows, dtype=np.uint64))
    assert ctypes.sizeof(cv.cv_buf) == 16
    assert as_pairs(one_by_one, 3)[0] == rows[0] and as_pairs(one_by_one, 3)[2] == rows[2]
    assert as_pairs(tuples, 3) == rows == as_pairs(desc, 3)
    for bad in (np.zeros((3, 3), np.uint64), np.zeros(4, np.uint64)):
        with pytest.raises(ValueError):
            cv._bufs(bad)
    with pytest.raises(ValueError):
        cv._bufs([(1, 2, 3), (4, 5, 6)])
