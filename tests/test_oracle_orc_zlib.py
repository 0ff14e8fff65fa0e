"""Oracle pins for ORC compressed streams with zlib compression: hand-derived
fixtures, and streams framed here and checked against zlib as an
independent decoder of each body, every prefix and the sizes query."""
import zlib

import numpy as np
import pytest

import oracle
import synth
from helpers import case_bytes, load_golden

CASES = load_golden("orc_zlib.json")


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_orc_zlib_golden(case):
    exp = case.get("text", "").encode()
    cap = case.get("cap", len(exp))
    st, out = oracle.decode_chunk(oracle.FMT_ORC_ZLIB, case_bytes(case), cap)
    assert st == case["status"], case["why"]
    if st == 0:
        assert out == exp, case["why"]


def _zlib_reference(stream: bytes) -> bytes:
    """Walk the 3-byte headers and decode each body with zlib."""
    out, pos = [], 0
    while pos < len(stream):
        v = stream[pos] | stream[pos + 1] << 8 | stream[pos + 2] << 16
        body = stream[pos + 3: pos + 3 + (v >> 1)]
        out.append(body if v & 1 else zlib.decompressobj(-15).decompress(body))
        pos += 3 + (v >> 1)
    return b"".join(out)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("block", [1000, 4096, 65536])
def test_framed_streams_against_zlib(seed, block):
    data = synth.plaintext(seed, 0, 150_000).tobytes()
    stream = synth.orc_zlib_stream(data, block)
    assert _zlib_reference(stream) == data
    assert oracle.decode_chunk(oracle.FMT_ORC_ZLIB, stream, len(data)) == (0, data)


def test_stored_and_compressed_mix():
    """Uniform bytes do not compress: those blocks are stored as is."""
    rng = np.random.default_rng(5)
    data = (b"abc" * 30000) + rng.integers(0, 256, 70000, dtype=np.uint8).tobytes() + b"z" * 5000
    stream = synth.orc_zlib_stream(data, 16384)
    kinds = []
    pos = 0
    while pos < len(stream):
        v = stream[pos] | stream[pos + 1] << 8 | stream[pos + 2] << 16
        kinds.append(v & 1)
        pos += 3 + (v >> 1)
    assert 0 in kinds and 1 in kinds
    assert oracle.decode_chunk(oracle.FMT_ORC_ZLIB, stream, len(data)) == (0, data)


def test_every_prefix_truncated_or_underflow():
    data = synth.plaintext(9, 0, 20_000).tobytes()
    stream = synth.orc_zlib_stream(data, 3000)
    for k in range(0, len(stream), 7):
        st, _ = oracle.decode_chunk(oracle.FMT_ORC_ZLIB, stream[:k], len(data))
        assert st in (oracle.TRUNCATED, oracle.OUTPUT_UNDERFLOW), k


def test_sizes_and_column():
    w = synth.orc_zlib_column(4, total=2 * synth.MiB, keep_plain=True)
    n, st = oracle.sizes(oracle.FMT_ORC_ZLIB, w.comp, w.comp_off)
    assert (st == 0).all() and np.array_equal(n, np.diff(w.out_off))
    out, st = oracle.decode(oracle.FMT_ORC_ZLIB, w.comp, w.comp_off, w.out_off, threads=4)
    assert (st == 0).all() and np.array_equal(out[: w.out_bytes], w.plain)
