"""Oracle pins for ORC byte RLE and boolean RLE: hand-derived fixtures, the
closed form of every stream of up to two bytes, round trips through an
independent encoder, numpy's bit unpacking for the boolean expansion, and
the prefix property."""
import numpy as np
import pytest

import oracle
import synth
from helpers import byte_rle_encode, case_bytes, expected_byte_rle, load_golden

CASES = load_golden("byte_rle.json")


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_byte_rle_golden(case):
    exp = expected_byte_rle(case)
    cap = case.get("cap", len(exp))
    st, out = oracle.decode_chunk(case["format"], case_bytes(case), cap)
    assert st == case["status"], case["why"]
    if st == 0:
        assert out == exp, case["why"]


def test_all_streams_up_to_two_bytes():
    """Closed form from the format definition: [h] alone is a run without its
    byte, or literals without their bytes (TRUNCATED) -- unless h decodes to
    nothing, which no control byte does; [h, x] is h+3 copies of x for
    h < 128, the literal x for h = 0xff, and TRUNCATED otherwise."""
    assert oracle.decode_chunk(oracle.FMT_BYTE_RLE, b"", None) == (0, b"")
    for h in range(256):
        st, _ = oracle.decode_chunk(oracle.FMT_BYTE_RLE, bytes([h]), None)
        assert st == oracle.TRUNCATED
        for x in (0, 1, 0x7f, 0x80, 0xff, h):
            st, out = oracle.decode_chunk(oracle.FMT_BYTE_RLE, bytes([h, x]), None)
            if h < 128:
                assert (st, out) == (0, bytes([x]) * (h + 3))
            elif h == 0xff:
                assert (st, out) == (0, bytes([x]))
            else:
                assert st == oracle.TRUNCATED


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_round_trip_independent_encoder(seed):
    rng = np.random.default_rng(seed)
    for _ in range(40):
        n = int(rng.integers(0, 3000))
        # runs and noise: repeat random bytes a random number of times
        vals = rng.integers(0, 256, size=max(n // 4, 1), dtype=np.uint8)
        reps = rng.integers(1, 200, size=vals.size)
        data = np.repeat(vals, reps)[:n].tobytes()
        enc = byte_rle_encode(data)
        assert oracle.decode_chunk(oracle.FMT_BYTE_RLE, enc, len(data)) == (0, data)


def test_generator_round_trip():
    """The generator's streams decode to the bytes it drew."""
    w = synth.byte_rle_column(4, total=2 * synth.MiB, keep_plain=True)
    out, st = oracle.decode(oracle.FMT_BYTE_RLE, w.comp, w.comp_off, w.out_off, threads=4)
    assert (st == 0).all() and np.array_equal(out[: w.out_bytes], w.plain)


@pytest.mark.parametrize("n_bools", [1, 7, 8, 9, 63, 64, 65, 1000, 4096])
def test_bool_is_unpacked_byte_rle(n_bools):
    """Boolean RLE = byte RLE + most-significant-bit-first unpacking
    (numpy.unpackbits), truncated to the span."""
    rng = np.random.default_rng(n_bools)
    packed = np.repeat(rng.integers(0, 256, size=(n_bools + 7) // 8 // 3 + 1, dtype=np.uint8),
                       3)[: (n_bools + 7) // 8].tobytes()
    enc = byte_rle_encode(packed)
    st, out = oracle.decode_chunk(oracle.FMT_BOOL_RLE, enc, n_bools)
    assert st == 0
    assert out == np.unpackbits(np.frombuffer(packed, np.uint8))[:n_bools].tobytes()
    # one boolean more needs one more byte only at a byte boundary
    st2, _ = oracle.decode_chunk(oracle.FMT_BOOL_RLE, enc, n_bools + 1)
    assert st2 == (oracle.OUTPUT_UNDERFLOW if n_bools % 8 == 0 else 0)


def test_every_prefix_truncated_or_underflow():
    data = bytes([5] * 40 + list(range(60)) + [9] * 7 + [200])
    enc = byte_rle_encode(data)
    for k in range(len(enc)):
        st, _ = oracle.decode_chunk(oracle.FMT_BYTE_RLE, enc[:k], len(data))
        assert st in (oracle.TRUNCATED, oracle.OUTPUT_UNDERFLOW), k


def test_sizes():
    data = bytes([1, 2, 3] + [4] * 50)
    enc = byte_rle_encode(data)
    assert oracle.decode_chunk(oracle.FMT_BYTE_RLE, enc, None) == (0, data)
    n, st = oracle.sizes(oracle.FMT_BOOL_RLE, np.frombuffer(enc, np.uint8),
                         np.array([0, len(enc)], np.uint64))
    assert st[0] == 0 and n[0] == 8 * len(data)
