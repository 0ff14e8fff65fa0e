"""Oracle: plain single-threaded CPU decoders (C, see ``oracle.h``).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
CPU-baseline leg of the benchmark are the only callers.  The library's
product path never imports this package, and this package never imports the
library: the two share no code.

``build()`` compiles the C sources with gcc into ``oracle/_build/liboracle.so``;
``decode()`` / ``sizes()`` run the plain per-chunk loop over a chunked buffer,
optionally splitting the chunk range over host threads (the C loop itself is
single-threaded; ctypes releases the GIL while it runs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = ["rle_v1.c", "rle_v2.c", "inflate.c", "byte_rle.c", "orc_frames.c", "batch.c"]

# Status codes (numeric values shared with the library's per-chunk status).
OK, TRUNCATED, OUTPUT_OVERFLOW, OUTPUT_UNDERFLOW = 0, 1, 2, 3
BAD_HEADER, BAD_HUFFMAN, BAD_DISTANCE, BAD_STORED_LEN, BAD_SPAN = 4, 5, 6, 7, 8

FMT_RLE_V1_I64, FMT_RLE_V2_I64, FMT_DEFLATE, FMT_RLE_V1_U64, FMT_RLE_V2_U64 = 1, 2, 3, 4, 5
FMT_BYTE_RLE, FMT_BOOL_RLE, FMT_ORC_ZLIB = 6, 7, 8

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    if not force and os.path.exists(LIB_PATH):
        newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(HERE, "oracle.h")])
        if os.path.getmtime(LIB_PATH) >= newest:
            return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp] + srcs
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            u8p = ctypes.c_void_p
            L.oracle_decode_chunk.argtypes = [ctypes.c_int, u8p, ctypes.c_size_t, u8p,
                                              ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
            L.oracle_decode_chunk.restype = ctypes.c_int
            L.oracle_decode_range.argtypes = [ctypes.c_int, u8p, u8p, u8p, u8p, u8p, u8p,
                                              ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_decode_range.restype = None
            L.oracle_sizes_range.argtypes = [ctypes.c_int, u8p, u8p, u8p, u8p, u8p,
                                             ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_sizes_range.restype = None
            _lib = L
        return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


SIZE_MAX = (1 << 64) - 1


def decode_chunk(fmt: int, data: bytes, cap: int | None = None):
    """Decode one chunk.  ``cap=None`` sizes the stream first (no store), then
    decodes into exactly that many bytes.  Returns (status, bytes)."""
    L = lib()
    src = np.frombuffer(bytes(data) + b"\0", dtype=np.uint8)  # never a NULL pointer
    n_out = ctypes.c_size_t(0)
    if cap is None:
        st = L.oracle_decode_chunk(fmt, _ptr(src), len(data), None, SIZE_MAX, ctypes.byref(n_out))
        if st != OK:
            return st, b""
        cap = n_out.value
    out = np.zeros(cap + 1, dtype=np.uint8)
    st = L.oracle_decode_chunk(fmt, _ptr(src), len(data), _ptr(out), cap, ctypes.byref(n_out))
    return st, out[: min(n_out.value, cap)].tobytes()


def _ranges(n: int, threads: int):
    threads = max(1, min(threads, n))
    step = (n + threads - 1) // threads
    return [(i, min(n, i + step)) for i in range(0, n, step)]


def decode(fmt: int, comp: np.ndarray, comp_off: np.ndarray, out_off: np.ndarray,
           formats: np.ndarray | None = None, threads: int = 1):
    """Decode every chunk; returns (out bytes as uint8 array, status int32 array)."""
    L = lib()
    n = len(comp_off) - 1
    comp = np.ascontiguousarray(comp, dtype=np.uint8)
    comp_off = np.ascontiguousarray(comp_off, dtype=np.uint64)
    out_off = np.ascontiguousarray(out_off, dtype=np.uint64)
    if formats is not None:
        formats = np.ascontiguousarray(formats, dtype=np.uint8)
    out = np.zeros(int(out_off[-1]) + 1 if n else 1, dtype=np.uint8)
    status = np.zeros(max(n, 1), dtype=np.int32)
    if comp.size == 0:
        comp = np.zeros(1, dtype=np.uint8)

    def run(r):
        L.oracle_decode_range(fmt, _ptr(formats), _ptr(comp), _ptr(comp_off), _ptr(out),
                              _ptr(out_off), _ptr(status), r[0], r[1])

    if n:
        if threads <= 1:
            run((0, n))
        else:
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(run, _ranges(n, threads)))
    return out[: int(out_off[-1]) if n else 0], status[:n]


def sizes(fmt: int, comp: np.ndarray, comp_off: np.ndarray,
          formats: np.ndarray | None = None, threads: int = 1):
    """Decoded size of every chunk; returns (sizes uint64, status int32)."""
    L = lib()
    n = len(comp_off) - 1
    comp = np.ascontiguousarray(comp, dtype=np.uint8)
    if comp.size == 0:
        comp = np.zeros(1, dtype=np.uint8)
    comp_off = np.ascontiguousarray(comp_off, dtype=np.uint64)
    if formats is not None:
        formats = np.ascontiguousarray(formats, dtype=np.uint8)
    sz = np.zeros(max(n, 1), dtype=np.uint64)
    status = np.zeros(max(n, 1), dtype=np.int32)

    def run(r):
        L.oracle_sizes_range(fmt, _ptr(formats), _ptr(comp), _ptr(comp_off), _ptr(sz),
                             _ptr(status), r[0], r[1])

    if n:
        if threads <= 1:
            run((0, n))
        else:
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(run, _ranges(n, threads)))
    return sz[:n], status[:n]
