"""ORC byte RLE and boolean RLE on the GPU through the C ABI, bit-exact
against the oracle: columns with ragged chunk sizes, every stream of up to
two bytes, mutated streams with right and wrong spans, the sizes query, a
mixed batch and the host-to-host call."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from devutil import assert_parity, pack, run_batch, run_plain, run_sizes  # noqa: E402

THREADS = os.cpu_count() or 4
FMTS = [synth.BYTE_RLE, synth.BOOL_RLE]


@pytest.mark.parametrize("fmt", FMTS)
def test_column_ragged_chunks(fmt):
    rng = np.random.default_rng(fmt)
    sizes = [int(s) for s in rng.integers(0, 200_000, size=300)]
    sizes[5] = 0
    w = synth.build_chunks([fmt] * len(sizes), sizes, 21, name="byte_rle_ragged")
    got, st = run_plain(fmt, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert_parity(fmt, w.comp, w.comp_off, w.out_off, got, st, threads=THREADS)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("shift", [0, 1, 3])
def test_unaligned_output(fmt, shift):
    w = synth.build_chunks([fmt] * 20, [1000 + 37 * i for i in range(20)], 5)
    got, st = run_plain(fmt, w.comp, w.comp_off, w.out_off, out_shift=shift)
    assert_parity(fmt, w.comp, w.comp_off, w.out_off, got, st, threads=THREADS)


@pytest.mark.parametrize("fmt", FMTS)
def test_short_streams_exhaustive(fmt):
    """Every 1- and 2-byte stream, sized by the oracle (errors: a 64-byte
    span, so that the stream's own problem is what is seen)."""
    chunks = [bytes([h]) for h in range(256)] + \
             [bytes([h, x]) for h in range(256) for x in (0, 0x55, 0x80, 0xff)]
    comp, coff = pack(chunks)
    sz, sst = oracle.sizes(fmt, comp, coff)
    span = np.where(sst == 0, sz, 64).astype(np.uint64)
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum(span)
    got, st = run_plain(fmt, comp, coff, ooff)
    assert_parity(fmt, comp, coff, ooff, got, st, threads=THREADS)


@pytest.mark.parametrize("fmt", FMTS)
def test_mutated_streams_and_wrong_spans(fmt):
    w = synth.build_chunks([fmt] * 400, [3000] * 400, 33)
    comp = w.comp.copy()
    rng = np.random.default_rng(9)
    for c in range(w.n):
        a, b = int(w.comp_off[c]), int(w.comp_off[c + 1])
        if c % 3 == 0 and b > a:
            comp[a + int(rng.integers(0, b - a))] = rng.integers(0, 256)
    d = 16 if fmt == synth.BOOL_RLE else 5  # booleans: two whole bytes
    spans = np.diff(w.out_off).astype(np.int64)
    spans[1::7] += d
    spans[2::7] -= d
    ooff = np.zeros(w.n + 1, np.uint64)
    ooff[1:] = np.cumsum(spans)
    got, st = run_plain(fmt, comp, w.comp_off, ooff)
    est = assert_parity(fmt, comp, w.comp_off, ooff, got, st, threads=THREADS)
    assert set(np.unique(est)) >= {0, 2, 3}


@pytest.mark.parametrize("fmt", FMTS)
def test_sizes_query(fmt):
    w = synth.build_chunks([fmt] * 50, [777 * (i + 1) for i in range(50)], 2)
    sz, st = run_sizes(fmt, w.comp, w.comp_off)
    exp, est = oracle.sizes(fmt, w.comp, w.comp_off)
    assert np.array_equal(st, est[: w.n]) and np.array_equal(sz, exp[: w.n])


def test_batch_with_byte_and_bool_rle():
    rng = np.random.default_rng(4)
    fmts = rng.choice([synth.RLE_V1_I64, synth.RLE_V2_I64, synth.DEFLATE, synth.BYTE_RLE,
                       synth.BOOL_RLE], size=600)
    sizes = (rng.integers(1, 60, size=600) * 1024).tolist()
    w = synth.build_chunks(fmts, sizes, 8, name="batch_bytes")
    got, st = run_batch(w.formats, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert_parity(0, w.comp, w.comp_off, w.out_off, got, st, formats=w.formats, threads=THREADS)
