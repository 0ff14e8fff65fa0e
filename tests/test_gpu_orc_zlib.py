"""ORC compressed streams (zlib) on the GPU through the C ABI, bit-exact
against the oracle: golden fixtures, ragged columns with stored and
compressed blocks, short streams, mutated streams and wrong spans, the
sizes query and a mixed batch."""
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import case_bytes, load_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from devutil import assert_parity, pack, run_batch, run_plain, run_sizes  # noqa: E402

THREADS = os.cpu_count() or 4
FMT = synth.ORC_ZLIB


def test_golden():
    cases = load_golden("orc_zlib.json")
    chunks = [case_bytes(c) for c in cases]
    caps = [c.get("cap", len(c.get("text", "").encode())) for c in cases]
    comp, coff = pack(chunks)
    ooff = np.zeros(len(cases) + 1, np.uint64)
    ooff[1:] = np.cumsum(caps)
    got, st = run_plain(FMT, comp, coff, ooff)
    assert [int(s) for s in st] == [c["status"] for c in cases]
    assert_parity(FMT, comp, coff, ooff, got, st, threads=THREADS)


@pytest.mark.parametrize("block", [4096, 65536])
def test_column_ragged(block):
    rng = np.random.default_rng(block)
    datas = [synth.plaintext(7, c, int(rng.integers(0, 300_000))).tobytes() for c in range(120)]
    chunks = [synth.orc_zlib_stream(d, block) for d in datas]
    comp, coff = pack(chunks)
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum([len(d) for d in datas])
    got, st = run_plain(FMT, comp, coff, ooff)
    assert (st == 0).all()
    assert np.array_equal(got, np.frombuffer(b"".join(datas), np.uint8))


def test_short_streams():
    """Every header value below 64 with bodies of the header's length cut
    from a few byte patterns, plus every 1- and 2-byte stream."""
    chunks = [bytes([h]) for h in range(256)] + [bytes([h, x]) for h in range(256) for x in (0, 7)]
    for v in range(64):
        for fill in (b"\x00", b"\x4b\x04\x00", b"\xff"):
            body = (fill * 40)[: v >> 1]
            chunks.append(bytes([v, 0, 0]) + body)
    comp, coff = pack(chunks)
    sz, sst = oracle.sizes(FMT, comp, coff)
    span = np.where(sst == 0, sz, 64).astype(np.uint64)
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum(span)
    got, st = run_plain(FMT, comp, coff, ooff)
    assert_parity(FMT, comp, coff, ooff, got, st, threads=THREADS)


def test_mutated_streams_and_wrong_spans():
    w = synth.build_chunks([FMT] * 200, [20000] * 200, 44)
    comp = w.comp.copy()
    rng = np.random.default_rng(3)
    for c in range(w.n):
        a, b = int(w.comp_off[c]), int(w.comp_off[c + 1])
        if c % 3 == 0 and b > a:
            comp[a + int(rng.integers(0, b - a))] ^= 1 << int(rng.integers(0, 8))
    spans = np.diff(w.out_off).astype(np.int64)
    spans[1::7] += 3
    spans[2::7] -= 3
    ooff = np.zeros(w.n + 1, np.uint64)
    ooff[1:] = np.cumsum(spans)
    got, st = run_plain(FMT, comp, w.comp_off, ooff)
    est = assert_parity(FMT, comp, w.comp_off, ooff, got, st, threads=THREADS)
    assert (est == 0).any() and (est != 0).any()


def test_sizes_query():
    w = synth.build_chunks([FMT] * 40, [9000 * (i + 1) for i in range(40)], 6)
    sz, st = run_sizes(FMT, w.comp, w.comp_off)
    exp, est = oracle.sizes(FMT, w.comp, w.comp_off)
    assert np.array_equal(st, est[: w.n]) and np.array_equal(sz, exp[: w.n])


def test_batch_with_orc_zlib():
    rng = np.random.default_rng(12)
    fmts = rng.choice([synth.RLE_V2_I64, synth.DEFLATE, synth.ORC_ZLIB, synth.BYTE_RLE], size=300)
    sizes = (rng.integers(1, 200, size=300) * 1024).tolist()
    w = synth.build_chunks(fmts, sizes, 17, name="batch_orc")
    got, st = run_batch(w.formats, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert_parity(0, w.comp, w.comp_off, w.out_off, got, st, formats=w.formats, threads=THREADS)
