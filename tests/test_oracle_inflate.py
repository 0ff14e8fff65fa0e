"""Pins for the Deflate oracle against zlib, used here as an independent
decoder (and, for round trips, as the encoder of every block type and
strategy), plus edge cases of RFC 1951 Sec. 3.2."""
import itertools
import random
import zlib

import numpy as np
import pytest

import oracle
import synth

STRATEGIES = {"default": zlib.Z_DEFAULT_STRATEGY, "filtered": zlib.Z_FILTERED,
              "huffman_only": zlib.Z_HUFFMAN_ONLY, "rle": zlib.Z_RLE, "fixed": zlib.Z_FIXED}


def zlib_inflate(data: bytes):
    d = zlib.decompressobj(-15)
    try:
        out = d.decompress(data)
    except zlib.error:
        return False, b""
    return d.eof, out


def special_texts():
    rng = random.Random(11)
    blk = bytes(rng.getrandbits(8) for _ in range(32768))
    return {
        "empty": b"",
        "one": b"x",
        "byte_run": b"\x00" * 100000,
        "period3": b"abc" * 20000,
        "max_distance": blk + blk[:4096],   # matches exactly 32768 back
        "text": b"the quick brown fox jumps over the lazy dog. " * 500,
    }


@pytest.mark.parametrize("strategy", list(STRATEGIES))
@pytest.mark.parametrize("level", [0, 1, 6, 9])
def test_round_trip_levels_and_strategies(level, strategy):
    texts = dict(special_texts())
    for kind in (0, 1, 2):
        texts[f"synth{kind}"] = synth.plaintext(3, kind, 65536, kind).tobytes()
    for name, txt in texts.items():
        comp = synth.deflate_bytes(txt, level, STRATEGIES[strategy])
        st, out = oracle.decode_chunk(oracle.FMT_DEFLATE, comp, len(txt))
        assert st == 0 and out == txt, name


def test_round_trip_column():
    w = synth.deflate_column(2, total=4 << 20, keep_plain=True)
    out, st = oracle.decode(oracle.FMT_DEFLATE, w.comp, w.comp_off, w.out_off, threads=4)
    assert (st == 0).all() and np.array_equal(out, w.plain)


def test_stored_block_is_memcpy():
    rng = random.Random(3)
    for n in (0, 1, 100, 65535):
        txt = bytes(rng.getrandbits(8) for _ in range(n))
        comp = bytes([1, n & 0xFF, n >> 8, ~n & 0xFF, (~n >> 8) & 0xFF]) + txt
        st, out = oracle.decode_chunk(oracle.FMT_DEFLATE, comp, n)
        assert st == 0 and out == txt


def _agree(data: bytes):
    ok_z, out_z = zlib_inflate(data)
    st, out = oracle.decode_chunk(oracle.FMT_DEFLATE, data)
    assert (st == 0) == ok_z, (data.hex(), st)
    if ok_z:
        assert out == out_z


def test_all_one_and_two_byte_streams_agree_with_zlib():
    for n in (1, 2):
        for b in itertools.product(range(256), repeat=n):
            _agree(bytes(b))


def test_random_short_streams_agree_with_zlib():
    rng = random.Random(1234)
    for _ in range(20000):
        _agree(bytes(rng.getrandbits(8) for _ in range(rng.randint(3, 8))))


def test_mutated_streams_agree_with_zlib():
    """Bit flips, truncations and splices of valid streams of every block
    type reach deep into the dynamic-header and code paths."""
    rng = random.Random(99)
    seeds = []
    for kind in (0, 1, 2):
        txt = synth.plaintext(5, kind, 3000, kind).tobytes()
        for strat in STRATEGIES.values():
            seeds.append(synth.deflate_bytes(txt, 6, strat))
    seeds.append(synth.deflate_bytes(b"abc" * 300, 9))
    for base in seeds:
        for _ in range(400):
            data = bytearray(base)
            op = rng.random()
            if op < 0.6:
                for _ in range(rng.randint(1, 3)):
                    i = rng.randrange(len(data) * 8)
                    data[i // 8] ^= 1 << (i % 8)
            elif op < 0.8:
                data = data[: rng.randrange(len(data))]
            else:
                i = rng.randrange(len(data))
                data[i:i + 4] = bytes(rng.getrandbits(8) for _ in range(4))
            _agree(bytes(data))
