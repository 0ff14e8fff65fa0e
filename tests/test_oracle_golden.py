"""Oracle vs hand-derived golden streams (tests/golden/*.json)."""
import pytest

import oracle
from helpers import (case_bytes, case_cap, expected_deflate, expected_rle,
                     load_golden)

RLE_CASES = [("rle_v1.json", c) for c in load_golden("rle_v1.json")] + \
            [("rle_v2.json", c) for c in load_golden("rle_v2.json")]
DEFLATE_CASES = load_golden("deflate.json")


@pytest.mark.parametrize("src,case", RLE_CASES, ids=[f"{s}:{c['name']}" for s, c in RLE_CASES])
def test_rle_golden(src, case):
    exp = expected_rle(case)
    st, out = oracle.decode_chunk(case["format"], case_bytes(case), case_cap(case, exp))
    assert st == case["status"], case["why"]
    if st == 0:
        assert out == exp, case["why"]


@pytest.mark.parametrize("case", DEFLATE_CASES, ids=[c["name"] for c in DEFLATE_CASES])
def test_deflate_golden(case):
    exp = expected_deflate(case)
    st, out = oracle.decode_chunk(oracle.FMT_DEFLATE, case_bytes(case), case_cap(case, exp))
    assert st == case["status"], case["why"]
    if st == 0:
        assert out == exp, case["why"]


@pytest.mark.parametrize("case", DEFLATE_CASES, ids=[c["name"] for c in DEFLATE_CASES])
def test_deflate_golden_agrees_with_zlib(case):
    """The fixtures themselves are checked by an independent decoder."""
    import zlib
    d = zlib.decompressobj(-15)
    try:
        out = d.decompress(case_bytes(case))
        ok = d.eof
    except zlib.error:
        ok = False
    if case["status"] == 0:
        assert ok and out == expected_deflate(case)
    elif case["status"] in (2, 3):  # a valid stream checked against a wrong span
        assert ok
    else:
        assert not ok
