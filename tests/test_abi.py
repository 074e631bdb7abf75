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
    lib.cv_free(None)


def test_no_cpu_path_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_0901_1307_gb300 import cv

    with pytest.raises(cv.CVError) as e:
        cv.master_build([bytes(1024)])
    assert e.value.code == cv.CV_ENODEV
