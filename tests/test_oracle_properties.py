"""Property-based pins of the oracle (hypothesis; CPU only): on arbitrary small inputs built from
a few reusable sector and fragment shapes (so that matches, duplicates, fills and partial tails
are common), every oracle route equals a pure-Python statement of its definition."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import oracle  # noqa: E402
from test_oracle import as_list, py_match  # noqa: E402
from test_oracle_fragments import py_frag_match  # noqa: E402

SECTOR, FRAG = 512, 64


def pieces(unit):
    """Byte strings that are whole units of a few shapes, or ragged tails."""
    base = np.random.default_rng(0).integers(0, 256, 4 * unit, dtype=np.uint8)
    shapes = [base[:unit], base[unit:2 * unit], base[2 * unit:3 * unit], bytes(unit), b"\x41" * unit]
    shapes = [bytes(x) for x in shapes]
    near = bytearray(unit)
    near[-1] = 1
    shapes.append(bytes(near))
    one = st.sampled_from(shapes)
    tail = st.binary(min_size=0, max_size=unit - 1)
    return st.lists(st.one_of(one, one, one, tail), min_size=0, max_size=6).map(b"".join)


@settings(max_examples=60, deadline=None)
@given(image=pieces(SECTOR), files=st.lists(pieces(SECTOR), min_size=0, max_size=4))
def test_sector_routes_equal_definition(image, files):
    want = py_match(image, files)
    img = np.frombuffer(image, np.uint8)
    fl = [np.frombuffer(f, np.uint8) for f in files]
    assert as_list(oracle.match_brute(img, fl)) == want
    assert as_list(oracle.match_hash(img, fl)) == want
    for sig in (1, 2, 3):
        assert as_list(oracle.match_sig(img, fl, sig)) == want


@settings(max_examples=60, deadline=None)
@given(image=pieces(SECTOR), files=st.lists(pieces(SECTOR), min_size=1, max_size=3),
       base=st.integers(min_value=0, max_value=20))
def test_position_route_equals_filtered_definition(image, files, base):
    want = [t for t in py_match(image, files) if (t[0] - base) % 8 == t[2] % 8]
    got = oracle.match_position(np.frombuffer(image, np.uint8), [np.frombuffer(f, np.uint8) for f in files], base)
    assert as_list(got) == want


@settings(max_examples=60, deadline=None)
@given(image=st.tuples(st.integers(0, 3), pieces(FRAG)).map(lambda t: b"\x07" * t[0] + t[1]),
       files=st.lists(pieces(FRAG), min_size=0, max_size=3))
def test_fragment_routes_equal_definition(image, files):
    want = py_frag_match(image, files)
    img = np.frombuffer(image, np.uint8)
    fl = [np.frombuffer(f, np.uint8) for f in files]
    assert as_list(oracle.frag_match_brute(img, fl)) == want
    assert as_list(oracle.frag_match(img, fl)) == want
