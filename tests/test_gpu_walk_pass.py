"""The RLE v2 walk pass (codag_set_walk_pass): segment starts found by a
separate launch that walks every chunk at once, against the walk inside each
decode CTA and against the oracle, bit-exact, on valid, mutated and
truncated streams, under several warps-per-chunk settings and through the
host-to-host entry point."""
import random

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from devutil import assert_parity, pack, run_plain  # noqa: E402
import paper_2307_03760_gb300 as codag  # noqa: E402

FMT = 2


@pytest.fixture(params=[0, 1], ids=["walk_in_cta", "walk_pass"])
def walk(request):
    assert codag.codag_get_walk_pass(FMT) == 0  # the default
    codag.codag_set_walk_pass(FMT, request.param)
    yield request.param
    codag.codag_set_walk_pass(FMT, 0)


@pytest.fixture(params=[2, 6, 16], ids=["parts_2", "parts_6", "parts_16"])
def parts(request):
    codag.codag_set_parts_per_chunk(request.param)
    yield request.param
    codag.codag_set_parts_per_chunk(0)


def test_column_both_walks(walk, parts):
    """A 16 MiB column of 128 KiB chunks (16 segments of 1024 values each)
    plus ragged chunk sizes (several tiles and a ragged tail)."""
    w = synth.rle_v2_column(seed=71, total=16 * synth.MiB)
    got, st = run_plain(FMT, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert_parity(FMT, w.comp, w.comp_off, w.out_off, got, st)
    r = synth.build_chunks([FMT] * 97, [8 * (1000 + 613 * k) for k in range(97)], seed=72)
    got, st = run_plain(FMT, r.comp, r.comp_off, r.out_off)
    assert (st == 0).all()
    assert_parity(FMT, r.comp, r.comp_off, r.out_off, got, st)


def test_mutated_long_chunks_both_walks(walk, parts):
    """Errors inside chunks long enough for many segments: the first error
    in stream order wins whichever segment finds it."""
    rng = random.Random(73)
    base = synth.build_chunks([FMT] * 6, [8 * 20000] * 6, seed=74)
    chunks = []
    for c in range(base.n):
        src = base.comp[int(base.comp_off[c]):int(base.comp_off[c + 1])].tobytes()
        for _ in range(40):
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
    sz, sst = oracle.sizes(FMT, comp, coff)
    caps = np.where(sst == 0, sz, 8 * 20000).astype(np.int64)
    caps = np.where(np.arange(len(chunks)) % 4 == 3, caps + 8, caps)
    ooff = np.zeros(len(chunks) + 1, np.uint64)
    ooff[1:] = np.cumsum(caps)
    got, st = run_plain(FMT, comp, coff, ooff)
    est = assert_parity(FMT, comp, coff, ooff, got, st)
    assert (est != 0).any() and (est == 0).any()


def test_walks_agree_on_every_prefix():
    """Every prefix of a 12,000-value chunk: both walks give the oracle's
    statuses and bytes."""
    w = synth.build_chunks([FMT], [8 * 12000], seed=75)
    src = w.comp.tobytes()
    chunks = [src[:k] for k in range(0, len(src) + 1, 7)] + [src]
    comp, coff = pack(chunks)
    full = int(w.out_off[-1])
    ooff = np.arange(len(chunks) + 1, dtype=np.uint64) * full
    codag.codag_set_parts_per_chunk(6)
    try:
        res = []
        for mode in (0, 1):
            codag.codag_set_walk_pass(FMT, mode)
            got, st = run_plain(FMT, comp, coff, ooff)
            assert_parity(FMT, comp, coff, ooff, got, st)
            res.append((got, st))
    finally:
        codag.codag_set_walk_pass(FMT, 0)
        codag.codag_set_parts_per_chunk(0)
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][0], res[1][0])
    assert res[1][1][-1] == 0


def test_walk_pass_through_host_entry_point(walk):
    w = synth.rle_v2_column(seed=76, total=48 * synth.MiB)
    h_out = np.zeros(w.out_bytes, np.uint8)
    h_st = np.full(w.n, -1, np.int32)
    d_comp = torch.zeros(w.comp_bytes + 16, dtype=torch.uint8, device="cuda:0")
    d_out = torch.zeros(w.out_bytes + 16, dtype=torch.uint8, device="cuda:0")
    codag.codag_decompress_host(FMT, w.comp, w.comp_off, w.n, h_out, w.out_off, d_comp, d_out, h_st)
    torch.cuda.synchronize()
    assert (h_st == 0).all()
    assert_parity(FMT, w.comp, w.comp_off, w.out_off, h_out, h_st)
