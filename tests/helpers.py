"""Shared test helpers: golden fixtures and tiny independent encoders.

The encoders here are written separately from the generator module and
from both decoders; they only produce inputs for brute-force checks.
"""
from __future__ import annotations

import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MASK64 = (1 << 64) - 1


def load_golden(name: str):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)["cases"]


def case_bytes(case) -> bytes:
    return bytes.fromhex(case["hex"].replace(" ", ""))


def expected_rle(case) -> bytes:
    """Expected little-endian 64-bit output of an RLE golden case."""
    vals = []
    if "values" in case:
        vals = list(case["values"])
    elif "fill" in case:
        for v, k in case["fill"]:
            vals += [v] * k
    elif "range" in case:
        vals = list(range(*case["range"]))
    return b"".join(((v & MASK64).to_bytes(8, "little")) for v in vals)


def expected_byte_rle(case) -> bytes:
    """Expected output of a byte / boolean RLE golden case."""
    if "bits" in case:
        return bytes(int(b) for b in case["bits"])
    if "fill_bytes" in case:
        return b"".join(bytes([v]) * k for v, k in case["fill_bytes"])
    return bytes.fromhex(case.get("out_hex", "").replace(" ", ""))


def byte_rle_encode(data: bytes) -> bytes:
    """Independent greedy ORC byte RLE encoder (runs of >= 3 equal bytes,
    everything else in literal groups of up to 128), for round trips."""
    out = bytearray()
    lit = bytearray()
    i, n = 0, len(data)

    def flush():
        while lit:
            k = min(len(lit), 128)
            out.append(256 - k)
            out.extend(lit[:k])
            del lit[:k]

    while i < n:
        j = i
        while j < n and j - i < 130 and data[j] == data[i]:
            j += 1
        if j - i >= 3:
            flush()
            out.append(j - i - 3)
            out.append(data[i])
            i = j
        else:
            lit.append(data[i])
            i += 1
    flush()
    return bytes(out)


def expected_deflate(case) -> bytes:
    if "text" in case:
        return case["text"].encode()
    if "fill_byte" in case:
        b, k = case["fill_byte"]
        return bytes([b]) * k
    return b""


def case_cap(case, expected: bytes) -> int:
    """Output span for a case: explicit, else the expected size for a valid
    stream, else a large span so the stream's own error is what is seen."""
    if "cap" in case:
        return case["cap"]
    return len(expected) if case["status"] == 0 else 1 << 20


# ---------------------------------------------------------------- encoders
def varint(u: int) -> bytes:
    out = bytearray()
    u &= MASK64
    while u >= 0x80:
        out.append((u & 0x7F) | 0x80)
        u >>= 7
    out.append(u)
    return bytes(out)


def zigzag(v: int) -> int:
    return ((v << 1) ^ (v >> 63)) & MASK64


def v1_literal(vals, signed: bool) -> bytes:
    assert 1 <= len(vals) <= 128
    return bytes([256 - len(vals)]) + b"".join(varint(zigzag(v) if signed else v) for v in vals)


def v1_run(base: int, delta: int, n: int, signed: bool) -> bytes:
    assert 3 <= n <= 130 and -128 <= delta <= 127
    return bytes([n - 3, delta & 0xFF]) + varint(zigzag(base) if signed else base)


def pack_msb(vals, width: int) -> bytes:
    bits = "".join(format(v & ((1 << width) - 1), f"0{width}b") for v in vals)
    bits += "0" * (-len(bits) % 8)
    return bytes(int(bits[i:i + 8], 2) for i in range(0, len(bits), 8))


WIDTHS = list(range(1, 25)) + [26, 28, 30, 32, 40, 48, 56, 64]


def v2_direct(vals_u, width: int) -> bytes:
    code = WIDTHS.index(width)
    n = len(vals_u)
    return bytes([0x40 | (code << 1) | ((n - 1) >> 8), (n - 1) & 0xFF]) + pack_msb(vals_u, width)


def to_signed(u: int) -> int:
    u &= MASK64
    return u - (1 << 64) if u >> 63 else u


def le64(vals) -> bytes:
    return b"".join((v & MASK64).to_bytes(8, "little") for v in vals)
