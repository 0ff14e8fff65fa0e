"""GPU path (through the C ABI) vs the oracle, bit-exact.

Every test runs the library's CUDA kernels and compares per-chunk status and
output bytes with the oracle on the same seeded inputs."""
import random

import numpy as np
import pytest

import oracle
import synth
from helpers import case_bytes, case_cap, expected_deflate, expected_rle, load_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from devutil import assert_parity, pack, run_batch, run_plain, run_sizes  # noqa: E402
import paper_2307_03760_gb300 as codag  # noqa: E402

RLE_FMTS = [1, 2, 4, 5]
ALL_FMTS = [1, 2, 3, 4, 5]


def _golden_by_format():
    groups = {}
    for name in ("rle_v1.json", "rle_v2.json"):
        for c in load_golden(name):
            groups.setdefault(c["format"], []).append((c, expected_rle(c)))
    for c in load_golden("deflate.json"):
        groups.setdefault(3, []).append((c, expected_deflate(c)))
    return groups


@pytest.mark.parametrize("fmt", [1, 2, 3, 4, 5])
def test_golden_fixtures(fmt):
    cases = _golden_by_format().get(fmt, [])
    if not cases:
        pytest.skip("no fixtures")
    chunks = [case_bytes(c) for c, _ in cases]
    caps = [case_cap(c, e) for c, e in cases]
    comp, coff = pack(chunks)
    ooff = np.zeros(len(caps) + 1, np.uint64)
    ooff[1:] = np.cumsum(caps)
    got, st = run_plain(fmt, comp, coff, ooff)
    for k, (c, e) in enumerate(cases):
        assert st[k] == c["status"], (c["name"], st[k])
        if c["status"] == 0:
            a = int(ooff[k])
            assert got[a:a + len(e)].tobytes() == e, c["name"]
    assert_parity(fmt, comp, coff, ooff, got, st)


@pytest.mark.parametrize("fmt", ALL_FMTS)
def test_workload_parity_small(fmt, parts):
    """Several chunks per SM tile plus ragged chunk sizes."""
    if fmt == 3 and parts:
        pytest.skip("parts apply to RLE only")
    if fmt == 3:
        sizes = [65536] * 40 + [1, 7, 100, 4095, 4096, 4097, 70000, 131072]
    else:
        base = 65536 if fmt in (1, 4) else 131072
        sizes = [base] * 40 + [8, 16, 24, 800, 4088, 8 * 513, 8 * 9999]
    w = synth.build_chunks([fmt] * len(sizes), sizes, seed=21 + fmt, keep_plain=True)
    got, st = run_plain(fmt, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert np.array_equal(got, w.plain)
    assert_parity(fmt, w.comp, w.comp_off, w.out_off, got, st)


@pytest.mark.parametrize("limit", [64 << 10, 1 << 20])
def test_deflate_pool_bound_fallback(limit):
    """A bounded command pool leaves the chunks past it to the one-warp
    decoder in the same call: every chunk must still match the oracle, for
    valid and for corrupted chunks."""
    sizes = [65536] * 12 + [1, 100, 4097, 70000, 131072, 300000]
    w = synth.build_chunks([3] * len(sizes), sizes, seed=41, keep_plain=True)
    comp = w.comp.copy()
    rng = np.random.default_rng(9)
    for c in range(2, w.n, 4):
        a, b = int(w.comp_off[c]), int(w.comp_off[c + 1])
        if b - a > 8:
            comp[rng.integers(a + 4, b)] ^= 0x21
    codag.codag_set_deflate_pool_limit(limit)
    try:
        got, st = run_plain(3, comp, w.comp_off, w.out_off)
    finally:
        codag.codag_set_deflate_pool_limit(0)
    assert_parity(3, comp, w.comp_off, w.out_off, got, st)
    assert (st == 0).sum() >= w.n // 2


def test_deflate_long_chunks_beside_short_ones():
    """Chunks whose output span is over 128 KiB go to the one-warp decoder
    after the two passes; those at or under it stay in the passes."""
    sizes = [4096, 131072, 131073, 700000, 65536, 131072 + 4096, 1000, 300000]
    w = synth.build_chunks([3] * len(sizes), sizes, seed=91)
    got, st = run_plain(3, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert_parity(3, w.comp, w.comp_off, w.out_off, got, st)
    # the sizes pass leaves chunks of over 64 KiB compressed to one warp
    sz, sst = run_sizes(3, w.comp, w.comp_off)
    assert (sst == 0).all() and np.array_equal(sz, np.array(sizes, np.uint64))


@pytest.mark.parametrize("shift", [1, 3, 8, 15])
def test_deflate_unaligned_output(shift):
    sizes = [65536, 1, 333, 65535, 20000]
    w = synth.build_chunks([3] * len(sizes), sizes, seed=5, keep_plain=True)
    got, st = run_plain(3, w.comp, w.comp_off, w.out_off, out_shift=shift)
    assert (st == 0).all() and np.array_equal(got, w.plain)


@pytest.mark.parametrize("level", [0, 1, 9])
@pytest.mark.parametrize("strategy", ["default", "filtered", "huffman_only", "rle", "fixed"])
def test_deflate_levels_and_strategies(level, strategy):
    import zlib
    strat = {"default": zlib.Z_DEFAULT_STRATEGY, "filtered": zlib.Z_FILTERED,
             "huffman_only": zlib.Z_HUFFMAN_ONLY, "rle": zlib.Z_RLE, "fixed": zlib.Z_FIXED}[strategy]
    texts = [synth.plaintext(8, k, 65536, k % 3).tobytes() for k in range(6)]
    rng = random.Random(4)
    blk = bytes(rng.getrandbits(8) for _ in range(32768))
    texts += [b"\x00" * 70000, b"abc" * 20000, blk + blk[:5000], b"", b"q"]
    chunks = [synth.deflate_bytes(t, level, strat) for t in texts]
    comp, coff = pack(chunks)
    ooff = np.zeros(len(texts) + 1, np.uint64)
    ooff[1:] = np.cumsum([len(t) for t in texts])
    got, st = run_plain(3, comp, coff, ooff)
    assert (st == 0).all()
    assert got.tobytes() == b"".join(texts)


@pytest.mark.parametrize("fmt", ALL_FMTS)
def test_sizes_query(fmt):
    sizes = [65536, 8, 4096, 131072, 0] if fmt != 3 else [65536, 1, 4096, 131072, 0]
    w = synth.build_chunks([fmt] * len(sizes), sizes, seed=31)
    got, st = run_sizes(fmt, w.comp, w.comp_off)
    exp, est = oracle.sizes(fmt, w.comp, w.comp_off)
    assert (st == est).all() and (got == exp).all()
    assert (got == np.diff(w.out_off)).all()


@pytest.mark.parametrize("fmt", ALL_FMTS)
def test_short_streams_exhaustive(fmt):
    """Every 1- and 2-byte stream: status (and output when OK) as the oracle.
    The output span is the oracle's decoded size when it has one."""
    chunks = [bytes([a]) for a in range(256)] + [bytes([a, b]) for a in range(256) for b in range(256)]
    comp, coff = pack(chunks)
    sz, sst = oracle.sizes(fmt, comp, coff)
    caps = np.where(sst == 0, sz, 64).astype(np.uint64)
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum(caps)
    got, st = run_plain(fmt, comp, coff, ooff)
    assert_parity(fmt, comp, coff, ooff, got, st)
    gsz, gst = run_sizes(fmt, comp, coff)
    assert (gst == sst).all()
    assert (gsz[sst == 0] == sz[sst == 0]).all()


@pytest.fixture(params=[0, 1, 6, 16], ids=["parts_auto", "parts_1", "parts_6", "parts_16"])
def parts(request):
    """Plain RLE calls split every chunk into this many warp-decoded parts."""
    import paper_2307_03760_gb300 as codag
    codag.codag_set_parts_per_chunk(request.param)
    yield request.param
    codag.codag_set_parts_per_chunk(0)


@pytest.mark.parametrize("fmt", ALL_FMTS)
def test_mutated_streams(fmt, parts):
    """Bit flips, truncations and splices of valid chunks; the chunk status
    combined over parts must still be the first error in stream order."""
    if fmt == 3 and parts:
        pytest.skip("parts apply to RLE only")
    rng = random.Random(100 + fmt)
    base = synth.build_chunks([fmt] * 8, [4096 if fmt != 3 else 5000] * 8, seed=41)
    chunks = []
    for c in range(base.n):
        src = base.comp[int(base.comp_off[c]):int(base.comp_off[c + 1])].tobytes()
        for _ in range(300):
            d = bytearray(src)
            op = rng.random()
            if op < 0.6:
                for _ in range(rng.randint(1, 3)):
                    i = rng.randrange(len(d) * 8)
                    d[i // 8] ^= 1 << (i % 8)
            elif op < 0.8:
                d = d[: rng.randrange(len(d))]
            else:
                i = rng.randrange(len(d))
                d[i:i + 4] = bytes(rng.getrandbits(8) for _ in range(4))
            chunks.append(bytes(d))
    comp, coff = pack(chunks)
    sz, sst = oracle.sizes(fmt, comp, coff)
    # half of the spans are the decoded size, the rest deliberately wrong
    caps = np.where(sst == 0, sz, 4096).astype(np.int64)
    flip = np.arange(len(chunks)) % 4 == 3
    caps = np.where(flip, caps + (8 if fmt != 3 else 1), caps)
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum(caps)
    got, st = run_plain(fmt, comp, coff, ooff)
    est = assert_parity(fmt, comp, coff, ooff, got, st)
    assert (est != 0).any() and (est == 0).any()


@pytest.mark.parametrize("fmt", [1, 2, 3])
def test_every_prefix_of_a_chunk(fmt, parts):
    if fmt == 3 and parts:
        pytest.skip("parts apply to RLE only")
    w = synth.build_chunks([fmt], [8 * 700 if fmt != 3 else 3000], seed=51)
    src = w.comp.tobytes()
    chunks = [src[:k] for k in range(len(src) + 1)]
    comp, coff = pack(chunks)
    full = int(w.out_off[-1])
    ooff = np.arange(len(chunks) + 1, dtype=np.uint64) * full
    got, st = run_plain(fmt, comp, coff, ooff)
    assert_parity(fmt, comp, coff, ooff, got, st)
    assert st[-1] == 0


@pytest.mark.parametrize("fmt", RLE_FMTS)
def test_rle_bad_spans(fmt):
    w = synth.build_chunks([fmt] * 3, [800, 800, 800], seed=61)
    ooff = np.array([0, 800, 1604, 2404], np.uint64)  # second span 804, third starts unaligned
    got, st = run_plain(fmt, w.comp, w.comp_off, ooff)
    assert st[0] == 0 and st[1] == oracle.BAD_SPAN and st[2] == oracle.BAD_SPAN


def test_empty_chunks_and_offsets():
    for fmt in ALL_FMTS:
        comp, coff = pack([b"", b"", b""])
        ooff = np.zeros(4, np.uint64)
        got, st = run_plain(fmt, comp, coff, ooff)
        exp = oracle.decode(fmt, comp, coff, ooff)[1]
        assert (st == exp).all()


def test_batch_mixed_and_graph():
    """Includes chunks up to 1 MiB, which the batch kernel splits into parts."""
    w = synth.batched(seed=3, n_chunks=600, lo=512, hi=1 << 20, keep_plain=True)
    got, st = run_batch(w.formats, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all() and np.array_equal(got, w.plain)
    got2, st2 = run_batch(w.formats, w.comp, w.comp_off, w.out_off, graph=True, replays=3)
    assert (st2 == 0).all() and np.array_equal(got2, w.plain)


SPLITS = [(16, 16), (12, 32), (14, 4), (16, 1)]


@pytest.mark.parametrize("split", SPLITS, ids=lambda s: f"split{s[0]}max{s[1]}")
def test_batch_every_staging_shape_and_split(split):
    """Every compiled input-ring shape of the batch kernel, under several RLE
    split rules (fine, coarse, never), decodes every chunk to the same bytes;
    also through a graph captured with the non-default choices."""
    shapes = codag.codag_batch_staging_shapes()
    assert len(shapes) >= 4 and (1024, 4) in shapes
    w = synth.batched(seed=5, n_chunks=300, lo=512, hi=1 << 20, keep_plain=True)
    try:
        codag.codag_set_batch_split(*split)
        for slot, slots in shapes:
            codag.codag_set_batch_staging(slot, slots)
            got, st = run_batch(w.formats, w.comp, w.comp_off, w.out_off)
            assert (st == 0).all(), (slot, slots)
            assert np.array_equal(got, w.plain), (slot, slots)
        got, st = run_batch(w.formats, w.comp, w.comp_off, w.out_off, graph=True, replays=2)
        assert (st == 0).all() and np.array_equal(got, w.plain)
    finally:
        codag.codag_set_batch_staging(0, 0)
        codag.codag_set_batch_split(0, 0)


@pytest.mark.parametrize("shape", [(256, 8), (2048, 4)])
def test_batch_errors_non_default_shape(shape):
    """Corrupted and truncated chunks give the oracle's statuses with a
    non-default ring shape and fine RLE splitting (errors inside parts)."""
    w = synth.batched(seed=8, n_chunks=96, lo=512, hi=1 << 20)
    comp = w.comp.copy()
    rng = np.random.default_rng(9)
    for c in range(1, w.n, 4):
        a, b = int(w.comp_off[c]), int(w.comp_off[c + 1])
        if b > a:
            comp[rng.integers(a, b)] ^= 0x33
    try:
        codag.codag_set_batch_staging(*shape)
        codag.codag_set_batch_split(12, 32)
        got, st = run_batch(w.formats, comp, w.comp_off, w.out_off)
    finally:
        codag.codag_set_batch_staging(0, 0)
        codag.codag_set_batch_split(0, 0)
    assert_parity(0, comp, w.comp_off, w.out_off, got, st, formats=w.formats)


def test_batch_unknown_format_and_errors():
    w = synth.batched(seed=4, n_chunks=64, lo=512, hi=1 << 20)
    fm = w.formats.copy()
    fm[5] = 9
    comp = w.comp.copy()
    rng = np.random.default_rng(7)
    for c in range(6, w.n, 3):  # corrupt a byte in every third chunk, big ones included
        a, b = int(w.comp_off[c]), int(w.comp_off[c + 1])
        if b > a:
            comp[rng.integers(a, b)] ^= 0x5A
    got, st = run_batch(fm, comp, w.comp_off, w.out_off)
    assert st[5] == oracle.BAD_HEADER
    fm2 = fm.copy()
    fm2[5] = 3  # the oracle needs a valid id; chunk 5 is compared separately
    exp, est = oracle.decode(0, comp, w.comp_off, w.out_off, formats=fm2)
    mask = np.arange(w.n) != 5
    assert (st[mask] == est[mask]).all()
    # the chunks left OK next to corrupted ones decode to the oracle's bytes
    ok = np.nonzero((est == 0) & mask)[0]
    assert ok.size > w.n // 3
    for c in ok:
        a, b = int(w.out_off[c]), int(w.out_off[c + 1])
        assert np.array_equal(got[a:b], exp[a:b]), f"chunk {c} differs"
