"""Seeded synthetic workloads (input generation only; no decoding arithmetic).

Builds the chunked inputs for the five workloads the library is measured on
and the tests check, using the C generators/encoders in ``synth.c`` and the
host zlib (``zlib.compressobj(level, DEFLATED, -15)``, i.e. raw Deflate) for
the Deflate chunks.  Everything is a pure function of ``seed``.

A workload is a ``Chunked`` record in the library's argument layout:
``comp`` (uint8), ``comp_off`` (uint64, n+1), ``out_off`` (uint64, n+1),
``formats`` (uint8 per chunk) and, when asked for, the expected plaintext /
values (``plain``) that produced it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import zlib
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libsynth.so")

RLE_V1_I64, RLE_V2_I64, DEFLATE, RLE_V1_U64, RLE_V2_U64 = 1, 2, 3, 4, 5
BYTE_RLE, BOOL_RLE, ORC_ZLIB = 6, 7, 8
FORMAT_NAMES = {1: "rle_v1", 2: "rle_v2", 3: "deflate", 4: "rle_v1_u64", 5: "rle_v2_u64"}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    src = os.path.join(HERE, "synth.c")
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(src):
        return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, src])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            for name in ("synth_rle_v1_chunk", "synth_rle_v2_chunk"):
                f = getattr(L, name)
                f.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]
                f.restype = ctypes.c_uint64
            L.synth_byte_rle_chunk.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]
            L.synth_byte_rle_chunk.restype = ctypes.c_uint64
            L.synth_plaintext.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_uint64]
            L.synth_plaintext.restype = ctypes.c_int
            _lib = L
        return _lib


@dataclass
class Chunked:
    comp: np.ndarray       # uint8, concatenated compressed chunks
    comp_off: np.ndarray   # uint64[n+1]
    out_off: np.ndarray    # uint64[n+1]
    formats: np.ndarray    # uint8[n]
    plain: np.ndarray | None = None  # uint8, expected output (if kept)
    name: str = ""

    @property
    def n(self) -> int:
        return len(self.comp_off) - 1

    @property
    def comp_bytes(self) -> int:
        return int(self.comp_off[-1])

    @property
    def out_bytes(self) -> int:
        return int(self.out_off[-1])


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def rle_chunk(fmt: int, seed: int, chunk: int, n_values: int, keep_values: bool = True):
    """Encode one generated RLE chunk; returns (encoded bytes, values or None)."""
    L = lib()
    signed = 1 if fmt in (RLE_V1_I64, RLE_V2_I64) else 0
    fn = L.synth_rle_v1_chunk if fmt in (RLE_V1_I64, RLE_V1_U64) else L.synth_rle_v2_chunk
    vals = np.empty(max(n_values, 1), dtype=np.int64) if keep_values else None
    cap = 12 * n_values + 64
    while True:
        enc = np.empty(cap, dtype=np.uint8)
        used = fn(seed, chunk, signed, n_values, None if vals is None else vals.ctypes.data,
                  enc.ctypes.data, cap)
        if used <= cap:
            return enc[:used].copy(), (vals[:n_values] if vals is not None else None)
        cap = int(used)


def byte_rle_chunk(seed: int, chunk: int, n_bytes: int, keep_values: bool = True):
    """Encode one generated ORC byte RLE chunk; returns (encoded, bytes or None)."""
    L = lib()
    vals = np.empty(max(n_bytes, 1), dtype=np.uint8) if keep_values else None
    cap = 2 * n_bytes + 64
    while True:
        enc = np.empty(cap, dtype=np.uint8)
        used = L.synth_byte_rle_chunk(seed, chunk, n_bytes, None if vals is None else vals.ctypes.data,
                                      enc.ctypes.data, cap)
        if used <= cap:
            return enc[:used].copy(), (vals[:n_bytes] if vals is not None else None)
        cap = int(used)


def orc_frame(body: bytes, original: bool) -> bytes:
    """One ORC compression chunk: 3-byte little-endian header (length << 1 |
    original) and the body."""
    v = (len(body) << 1) | (1 if original else 0)
    return bytes((v & 0xFF, (v >> 8) & 0xFF, (v >> 16) & 0xFF)) + body


def orc_zlib_stream(data, block: int = 64 * 1024, level: int = 6) -> bytes:
    """An ORC compressed stream as an ORC writer makes it: the data cut into
    blocks, each compressed as raw Deflate, or stored as is when that is not
    smaller."""
    data = bytes(data)
    out = []
    for i in range(0, len(data), block):
        piece = data[i:i + block]
        comp = deflate_bytes(piece, level)
        out.append(orc_frame(comp, False) if len(comp) < len(piece) else orc_frame(piece, True))
    return b"".join(out)


def plaintext(seed: int, chunk: int, n: int, kind: int = -1) -> np.ndarray:
    out = np.empty(max(n, 1), dtype=np.uint8)
    lib().synth_plaintext(seed, chunk, kind, out.ctypes.data, n)
    return out[:n]


def deflate_bytes(data, level: int = 6, strategy: int = zlib.Z_DEFAULT_STRATEGY) -> bytes:
    c = zlib.compressobj(level, zlib.DEFLATED, -15, 8, strategy)
    return c.compress(bytes(data)) + c.flush()


def _assemble(parts, sizes, fmts, keep_plain, plains, name):
    n = len(parts)
    comp_off = np.zeros(n + 1, dtype=np.uint64)
    comp_off[1:] = np.cumsum([len(p) for p in parts], dtype=np.uint64) if n else []
    out_off = np.zeros(n + 1, dtype=np.uint64)
    out_off[1:] = np.cumsum(np.asarray(sizes, dtype=np.uint64), dtype=np.uint64) if n else []
    comp = np.concatenate(parts) if n else np.zeros(0, dtype=np.uint8)
    plain = None
    if keep_plain:
        plain = np.concatenate(plains) if n else np.zeros(0, dtype=np.uint8)
    return Chunked(comp.astype(np.uint8, copy=False), comp_off, out_off,
                   np.asarray(fmts, dtype=np.uint8), plain, name)


def build_chunks(fmts, sizes, seed: int, keep_plain: bool = False, level: int = 6,
                 strategy: int = zlib.Z_DEFAULT_STRATEGY, threads: int | None = None,
                 name: str = "") -> Chunked:
    """Generate chunk c of format fmts[c] with sizes[c] uncompressed bytes
    (RLE sizes must be multiples of 8)."""
    fmts = [int(f) for f in fmts]
    sizes = [int(s) for s in sizes]
    n = len(fmts)

    def one(c):
        f, s = fmts[c], sizes[c]
        if f == DEFLATE:
            p = plaintext(seed, c, s)
            return np.frombuffer(deflate_bytes(p, level, strategy), dtype=np.uint8), p
        if f == BYTE_RLE:
            return byte_rle_chunk(seed, c, s, keep_plain)
        if f == ORC_ZLIB:  # ORC stream of 64 KiB compression blocks
            p = plaintext(seed, c, s)
            return np.frombuffer(orc_zlib_stream(p, 64 * 1024, level), dtype=np.uint8), p
        if f == BOOL_RLE:  # s booleans: ceil(s / 8) packed bytes, expanded MSB first
            enc, packed = byte_rle_chunk(seed, c, (s + 7) // 8, keep_plain)
            return enc, (np.unpackbits(packed)[:s] if packed is not None else None)
        enc, vals = rle_chunk(f, seed, c, s // 8, keep_plain)
        return enc, (vals.view(np.uint8) if vals is not None else None)

    th = threads or _threads()
    if th > 1 and n > 1:
        with ThreadPoolExecutor(th) as ex:
            res = list(ex.map(one, range(n)))
    else:
        res = [one(c) for c in range(n)]
    parts = [r[0] for r in res]
    plains = [r[1] for r in res]
    return _assemble(parts, sizes, fmts, keep_plain, plains, name)


# --------------------------------------------------------------- workloads
MiB = 1 << 20
GiB = 1 << 30


def rle_v1_column(seed: int = 1, total: int = 8 * MiB, chunk: int = 64 * 1024, **kw) -> Chunked:
    """ORC RLE v1, signed int64: 8 MiB in 64 KiB chunks (128 chunks)."""
    n = total // chunk
    return build_chunks([RLE_V1_I64] * n, [chunk] * n, seed, name="rle_v1", **kw)


def rle_v2_column(seed: int = 1, total: int = 256 * MiB, chunk: int = 128 * 1024, **kw) -> Chunked:
    """ORC RLE v2, signed int64: 256 MiB in 128 KiB chunks (2048 chunks)."""
    n = total // chunk
    return build_chunks([RLE_V2_I64] * n, [chunk] * n, seed, name="rle_v2", **kw)


def deflate_column(seed: int = 1, total: int = 1 * GiB, chunk: int = 64 * 1024, **kw) -> Chunked:
    """Raw Deflate, zlib level 6: 1 GiB in 64 KiB chunks (16384 chunks)."""
    n = total // chunk
    return build_chunks([DEFLATE] * n, [chunk] * n, seed, name="deflate", **kw)


def byte_rle_column(seed: int = 1, total: int = 64 * MiB, chunk: int = 64 * 1024, **kw) -> Chunked:
    """ORC byte RLE: 64 MiB of bytes in 64 KiB chunks (1024 chunks)."""
    n = total // chunk
    return build_chunks([BYTE_RLE] * n, [chunk] * n, seed, name="byte_rle", **kw)


def bool_rle_column(seed: int = 1, total: int = 64 * MiB, chunk: int = 64 * 1024, **kw) -> Chunked:
    """ORC boolean RLE: 64 Mi booleans (one output byte each) in chunks of 64 Ki."""
    n = total // chunk
    return build_chunks([BOOL_RLE] * n, [chunk] * n, seed, name="bool_rle", **kw)


def orc_zlib_column(seed: int = 1, total: int = 1 * GiB, chunk: int = 256 * 1024, **kw) -> Chunked:
    """ORC zlib streams: 1 GiB as 4096 streams of 256 KiB, each four 64 KiB
    compression blocks (raw Deflate level 6, stored when not smaller)."""
    n = total // chunk
    return build_chunks([ORC_ZLIB] * n, [chunk] * n, seed, name="orc_zlib", **kw)


def batched_plan(seed: int = 1, n_chunks: int = 20000, lo: int = 4096, hi: int = MiB):
    """Mixed batch plan: 40% RLE v2, 20% RLE v1, 40% Deflate; sizes
    log-uniform in [lo, hi), rounded down to a multiple of 8 so that every
    chunk's output offset suits the 8-byte RLE values."""
    g = np.random.Generator(np.random.PCG64(seed * 7919 + 4))
    u = g.integers(0, 100, n_chunks)
    fmts = np.where(u < 40, RLE_V2_I64, np.where(u < 60, RLE_V1_I64, DEFLATE)).astype(np.uint8)
    lo_oct, hi_oct = int(np.log2(lo)), int(np.log2(hi))
    octave = g.integers(lo_oct, hi_oct, n_chunks)
    sizes = (np.left_shift(1, octave) + g.integers(0, 1 << 62, n_chunks) % np.left_shift(1, octave))
    sizes = (sizes // 8 * 8).astype(np.int64)
    return fmts, sizes


def batched(seed: int = 1, n_chunks: int = 20000, lo: int = 4096, hi: int = MiB, **kw) -> Chunked:
    fmts, sizes = batched_plan(seed, n_chunks, lo, hi)
    return build_chunks(fmts, sizes, seed, name="batched", **kw)


def serving_pool(seed: int = 1, n_payloads: int = 32, lo: int = 64 * 1024, hi: int = 64 * MiB,
                 keep_plain: bool = False, threads: int | None = None):
    """Request payloads for the serving workload: each a random format (RLE
    v1, RLE v2 or Deflate, uniform), total decoded size log-uniform in
    [lo, hi), 1-256 chunks of equal size (multiples of 8 bytes)."""
    g = np.random.Generator(np.random.PCG64(seed * 104729 + 5))
    pool = []
    for p in range(n_payloads):
        fmt = int(g.choice([RLE_V1_I64, RLE_V2_I64, DEFLATE]))
        total = int(np.exp(g.uniform(np.log(lo), np.log(hi))))
        n = int(g.integers(1, 257))
        size = max(8, total // n // 8 * 8)
        pool.append(build_chunks([fmt] * n, [size] * n, seed * 1000 + p, keep_plain=keep_plain,
                                 threads=threads, name=f"payload{p}"))
    return pool


def poisson_arrivals(seed: int, rate: float, duration: float, n_payloads: int):
    """Arrival times (seconds) of a Poisson process of `rate` requests/s over
    `duration` seconds, and the payload each request carries."""
    g = np.random.Generator(np.random.PCG64(seed * 7 + int(rate)))
    n = max(1, int(rate * duration * 1.5) + 16)
    t = np.cumsum(g.exponential(1.0 / rate, n))
    t = t[t < duration]
    return t, g.integers(0, n_payloads, len(t))
