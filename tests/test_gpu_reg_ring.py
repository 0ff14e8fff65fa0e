"""The register staging ring (codag_set_input_staging mode 1) for Deflate and
byte / boolean RLE: the same parity checks as with the shared-memory ring."""
import os
import random
import zlib

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2307_03760_gb300 as codag  # noqa: E402
from devutil import assert_parity, pack, run_plain  # noqa: E402

THREADS = os.cpu_count() or 4
FAMS = (synth.DEFLATE, synth.BYTE_RLE, synth.BOOL_RLE)


@pytest.fixture(autouse=True)
def register_ring():
    for f in FAMS:
        codag.codag_set_input_staging(f, 1)
    assert codag.codag_get_input_staging(synth.DEFLATE) == 1
    yield
    for f in FAMS:
        codag.codag_set_input_staging(f, 0)


@pytest.mark.parametrize("level", [0, 1, 6, 9])
@pytest.mark.parametrize("strategy", [zlib.Z_DEFAULT_STRATEGY, zlib.Z_HUFFMAN_ONLY, zlib.Z_RLE, zlib.Z_FIXED])
def test_deflate_levels_and_strategies(level, strategy):
    texts = [synth.plaintext(8, k, 65536, k % 3).tobytes() for k in range(6)]
    rng = random.Random(4)
    blk = bytes(rng.getrandbits(8) for _ in range(32768))
    texts += [b"\x00" * 70000, b"abc" * 20000, blk + blk[:5000], b"", b"q"]
    comp, coff = pack([synth.deflate_bytes(t, level, strategy) for t in texts])
    ooff = np.zeros(len(texts) + 1, np.uint64)
    ooff[1:] = np.cumsum([len(t) for t in texts])
    got, st = run_plain(synth.DEFLATE, comp, coff, ooff, out_shift=3)
    assert (st == 0).all() and got.tobytes() == b"".join(texts)


@pytest.mark.parametrize("fmt", FAMS)
def test_short_streams_exhaustive(fmt):
    chunks = [bytes([a]) for a in range(256)] + [bytes([a, b]) for a in range(256) for b in range(256)]
    comp, coff = pack(chunks)
    sz, sst = oracle.sizes(fmt, comp, coff)
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum(np.where(sst == 0, sz, 64).astype(np.uint64))
    got, st = run_plain(fmt, comp, coff, ooff)
    assert_parity(fmt, comp, coff, ooff, got, st)


@pytest.mark.parametrize("fmt", FAMS)
def test_mutated_streams_and_prefixes(fmt):
    rng = random.Random(7 + fmt)
    base = synth.build_chunks([fmt] * 6, [5000] * 6, seed=43)
    chunks = []
    for c in range(base.n):
        src = base.comp[int(base.comp_off[c]):int(base.comp_off[c + 1])].tobytes()
        chunks += [src[:k] for k in range(0, len(src) + 1, 17)]
        for _ in range(200):
            d = bytearray(src)
            for _ in range(rng.randint(1, 3)):
                i = rng.randrange(len(d) * 8)
                d[i // 8] ^= 1 << (i % 8)
            chunks.append(bytes(d))
    comp, coff = pack(chunks)
    ooff = np.arange(len(chunks) + 1, dtype=np.uint64) * 5000
    got, st = run_plain(fmt, comp, coff, ooff)
    assert_parity(fmt, comp, coff, ooff, got, st, threads=THREADS)


@pytest.mark.parametrize("fmt,total", [(synth.DEFLATE, 64 * synth.MiB), (synth.BYTE_RLE, 64 * synth.MiB),
                                       (synth.BOOL_RLE, 64 * synth.MiB)])
def test_columns(fmt, total):
    w = synth.build_chunks([fmt] * (total // 65536), [65536] * (total // 65536), 3)
    got, st = run_plain(fmt, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert_parity(fmt, w.comp, w.comp_off, w.out_off, got, st, threads=THREADS)
