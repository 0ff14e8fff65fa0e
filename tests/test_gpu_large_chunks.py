"""RLE chunks too large to be staged whole in shared memory (the plain
CTA-per-chunk kernels then walk them through a ring and decode one part per
warp), next to chunks that are staged: bit-exact against the oracle for
ORC RLE v1, RLE v2 and byte RLE, with every launch shape of the parity
suite, plus corrupted large chunks whose status must be the first error in
stream order, and chunks around the size where the widened stage ends."""
import numpy as np
import pytest

import oracle
import synth
from helpers import v1_literal, v2_direct

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2307_03760_gb300 as codag  # noqa: E402
from devutil import assert_parity, pack, run_plain  # noqa: E402

# above the largest dynamic shared memory of a CTA on any current GPU
BIG = 240 * 1024


def big_rle_v1(rng, size=BIG) -> bytes:
    """Literal groups of full-range values: about 9.3 bytes per value."""
    out = bytearray()
    while len(out) < size:
        vals = rng.integers(-(1 << 62), 1 << 62, size=128, dtype=np.int64)
        out += v1_literal([int(v) for v in vals], True)
    return bytes(out)


def big_rle_v2(rng, size=BIG) -> bytes:
    """DIRECT runs of 512 values at width 64 (8 bytes per value), with a
    narrower run now and then so that widths change along the chunk."""
    out = bytearray()
    k = 0
    while len(out) < size:
        w = 64 if k % 4 else 56
        vals = rng.integers(0, 1 << 62, size=512, dtype=np.uint64) & np.uint64((1 << w) - 1)
        out += v2_direct([int(v) for v in vals], w)
        k += 1
    return bytes(out)


def big_byte_rle(rng, size=BIG) -> bytes:
    """Literal groups of 128 random bytes (129 stream bytes each)."""
    out = bytearray()
    while len(out) < size:
        out.append(0x80)  # -128: 128 literal bytes
        out += rng.integers(0, 256, size=128, dtype=np.uint8).tobytes()
    return bytes(out)


MAKE = {synth.RLE_V1_I64: big_rle_v1, synth.RLE_V2_I64: big_rle_v2, synth.BYTE_RLE: big_byte_rle}


@pytest.fixture(params=[0, 1, 6, 16], ids=["parts_auto", "parts_1", "parts_6", "parts_16"])
def parts(request):
    codag.codag_set_parts_per_chunk(request.param)
    yield request.param
    codag.codag_set_parts_per_chunk(0)


def column(fmt, seed, corrupt=False):
    rng = np.random.default_rng(seed)
    small = synth.build_chunks([fmt] * 12, [65536] * 12, seed=seed)
    chunks = []
    for c in range(small.n):
        chunks.append(small.comp[int(small.comp_off[c]):int(small.comp_off[c + 1])].tobytes())
        if c % 4 == 1:
            b = bytearray(MAKE[fmt](rng))
            if corrupt and c % 8 == 1:
                b[len(b) // 2 + c] ^= 0x80  # deep inside: a later part sees it
            elif corrupt:
                del b[len(b) - 1000:]  # truncated deep inside the last run
            chunks.append(bytes(b))
    comp, coff = pack(chunks)
    sz, sst = oracle.sizes(fmt, comp, coff)
    span = np.where(sst == 0, sz, 1 << 16).astype(np.uint64)
    if fmt != synth.BYTE_RLE:
        span = (span + 7) // 8 * 8
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum(span)
    return comp, coff, ooff, sst


@pytest.mark.parametrize("fmt", sorted(MAKE))
def test_large_chunks_beside_staged_ones(fmt, parts):
    comp, coff, ooff, sst = column(fmt, 5 + fmt)
    assert (sst == 0).all()
    assert int(np.diff(coff.astype(np.int64)).max()) >= BIG
    got, st = run_plain(fmt, comp, coff, ooff)
    assert (st == 0).all()
    assert_parity(fmt, comp, coff, ooff, got, st)


@pytest.mark.parametrize("fmt", sorted(MAKE))
def test_corrupted_large_chunks(fmt, parts):
    comp, coff, ooff, sst = column(fmt, 9 + fmt, corrupt=True)
    got, st = run_plain(fmt, comp, coff, ooff)
    assert_parity(fmt, comp, coff, ooff, got, st)


@pytest.mark.parametrize("fmt", sorted(MAKE))
def test_chunks_around_the_stage_limit(fmt, parts):
    """Compressed sizes from 30 to 50 KiB: staged whole or streamed through
    rings, depending on the stage each launch shape gets."""
    rng = np.random.default_rng(77 + fmt)
    chunks = [MAKE[fmt](rng, size) for size in range(30 * 1024, 50 * 1024, 1536)]
    comp, coff = pack(chunks)
    sz, sst = oracle.sizes(fmt, comp, coff)
    assert (sst == 0).all()
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum(sz.astype(np.uint64))
    got, st = run_plain(fmt, comp, coff, ooff)
    assert (st == 0).all()
    assert_parity(fmt, comp, coff, ooff, got, st)
