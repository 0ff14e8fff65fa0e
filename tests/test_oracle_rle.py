"""Pins for the RLE oracles: brute force over tiny columns and every legal
encoding of them, round trips through the generator's independent encoder,
truncation and sizing invariants."""
import itertools
import random

import numpy as np
import pytest

import oracle
import synth
from helpers import (MASK64, WIDTHS, le64, pack_msb, to_signed, v1_literal,
                     v1_run, v2_direct)

SMALL = [-2, -1, 0, 1, 2, -(1 << 63), (1 << 63) - 1]


def _segmentations(n):
    """All compositions of n as tuples of part lengths."""
    if n == 0:
        yield ()
        return
    for first in range(1, n + 1):
        for rest in _segmentations(n - first):
            yield (first,) + rest


def _v1_encodings(seq, signed):
    """Every RLE v1 encoding of seq: each part a literal group or, when the
    part is an arithmetic sequence with an int8 step and 3+ values, a run."""
    for seg in _segmentations(len(seq)):
        parts, i = [], 0
        for ln in seg:
            part = seq[i:i + ln]
            opts = [v1_literal(part, signed)]
            if ln >= 3:
                d = to_signed((part[1] - part[0]) & MASK64)
                if -128 <= d <= 127 and all(((part[k] - part[0]) - k * d) & MASK64 == 0 for k in range(ln)):
                    base = part[0] if signed else part[0] & MASK64
                    opts.append(v1_run(base, d, ln, signed))
            parts.append(opts)
            i += ln
        for choice in itertools.product(*parts):
            yield b"".join(choice)


@pytest.mark.parametrize("signed", [True, False])
def test_rle_v1_brute_force_all_encodings(signed):
    fmt = oracle.FMT_RLE_V1_I64 if signed else oracle.FMT_RLE_V1_U64
    maxlen = 5 if signed else 4
    n_checked = 0
    for n in range(1, maxlen + 1):
        for seq in itertools.product(SMALL, repeat=n):
            seq = list(seq) if signed else [v & MASK64 for v in seq]
            exp = le64(seq)
            for enc in _v1_encodings(seq, signed):
                st, out = oracle.decode_chunk(fmt, enc, len(exp))
                assert st == 0 and out == exp, (seq, enc.hex())
                n_checked += 1
    assert n_checked > 1000


def test_rle_v2_direct_brute_force():
    """All values 0..2^w-1, in sequences of up to 3, at widths 1..4."""
    for w in (1, 2, 3, 4):
        for n in (1, 2, 3):
            for seq in itertools.product(range(1 << w), repeat=n):
                enc = v2_direct(list(seq), w)
                st, out = oracle.decode_chunk(oracle.FMT_RLE_V2_U64, enc, 8 * n)
                assert st == 0 and out == le64(seq), (w, seq)


@pytest.mark.parametrize("width", WIDTHS)
def test_rle_v2_direct_every_width(width):
    rng = random.Random(width)
    for n in (1, 7, 8, 9, 33, 512):
        vals = [rng.getrandbits(width) for _ in range(n)]
        vals[0] = (1 << width) - 1  # all ones at the top
        enc = v2_direct(vals, width)
        st, out = oracle.decode_chunk(oracle.FMT_RLE_V2_U64, enc, 8 * n)
        assert st == 0 and out == le64(vals)
        # signed columns zigzag DIRECT values
        st, out = oracle.decode_chunk(oracle.FMT_RLE_V2_I64, enc, 8 * n)
        assert st == 0 and out == le64([(v >> 1) ^ -(v & 1) for v in vals])


@pytest.mark.parametrize("fmt", [oracle.FMT_RLE_V1_I64, oracle.FMT_RLE_V2_I64,
                                 oracle.FMT_RLE_V1_U64, oracle.FMT_RLE_V2_U64])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rle_round_trip_generator(fmt, seed):
    """Generator + independent encoder -> oracle == generated values."""
    n_values = 8192 if fmt in (1, 4) else 16384
    w = synth.build_chunks([fmt] * 16, [8 * n_values] * 16, seed, keep_plain=True)
    out, st = oracle.decode(fmt, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert np.array_equal(out, w.plain)


def test_rle_v1_full_column_round_trip():
    w = synth.rle_v1_column(1, keep_plain=True)
    assert w.n == 128
    out, st = oracle.decode(1, w.comp, w.comp_off, w.out_off, threads=4)
    assert (st == 0).all() and np.array_equal(out, w.plain)


@pytest.mark.parametrize("fmt", [oracle.FMT_RLE_V1_I64, oracle.FMT_RLE_V2_I64])
def test_rle_prefix_truncation_and_sizes(fmt):
    """Every prefix of a valid chunk is either TRUNCATED (cut inside a group)
    or decodes to fewer values (cut at a group boundary), and sizing agrees
    with decoding."""
    enc, vals = synth.rle_chunk(fmt, 7, 0, 700)
    full = le64(vals.tolist())
    for cut in range(0, len(enc)):
        st, out = oracle.decode_chunk(fmt, enc[:cut].tobytes(), len(full))
        assert st in (oracle.TRUNCATED, oracle.OUTPUT_UNDERFLOW)
        sz, sst = oracle.sizes(fmt, enc[:cut], np.array([0, cut], np.uint64))
        if sst[0] == 0:
            assert st == oracle.OUTPUT_UNDERFLOW and sz[0] < len(full)
            st2, out2 = oracle.decode_chunk(fmt, enc[:cut].tobytes(), int(sz[0]))
            assert st2 == 0 and out2 == full[: int(sz[0])]
        else:
            assert sst[0] == st == oracle.TRUNCATED


def test_rle_v2_delta_invariants():
    """DELTA runs: monotone in the delta base's sign, count = sum of lengths."""
    rng = random.Random(5)
    for _ in range(300):
        n = rng.randint(3, 512)
        w = rng.choice([2, 3, 4, 8, 12, 16, 24])
        deltas = [rng.getrandbits(w) for _ in range(n - 2)]
        down = rng.random() < 0.5
        base = rng.randint(0, 1 << 40)
        d0 = rng.randint(1, 100) * (-1 if down else 1)
        code = WIDTHS.index(w)
        from helpers import varint, zigzag
        enc = bytes([0xC0 | (code << 1) | ((n - 1) >> 8), (n - 1) & 0xFF]) + varint(zigzag(base)) + \
            varint(zigzag(d0)) + pack_msb(deltas, w)
        st, out = oracle.decode_chunk(oracle.FMT_RLE_V2_I64, enc, 8 * n)
        assert st == 0
        v = np.frombuffer(out, dtype=np.int64)
        dv = np.diff(v)
        assert (dv <= 0).all() if down else (dv >= 0).all()
        assert v[0] == base and v[1] == base + d0
        assert np.array_equal(np.abs(dv[1:]), np.asarray(deltas, dtype=np.int64))


def test_all_short_streams_are_handled():
    """Every 1- and 2-byte stream decodes or reports an error code; sizing
    and decoding agree."""
    for fmt in (1, 2, 4, 5):
        for n in (1, 2):
            for b in itertools.product(range(256), repeat=n):
                data = bytes(b)
                st, out = oracle.decode_chunk(fmt, data)
                assert st in range(0, 9)
                if st == 0:
                    st2, out2 = oracle.decode_chunk(fmt, data, len(out))
                    assert st2 == 0 and out2 == out
