"""Python binding of libcodag.so: chunk-parallel GPU decompression of ORC
integer RLE v1/v2 and raw Deflate on one GB300 (CODAG, arXiv 2307.03760).

Argument marshalling only: every decoding step runs in the CUDA kernels
behind the C ABI declared in ``include/codag.h``; the functions here carry
the same names and turn torch tensors (device memory) and torch streams into
the raw pointers and stream handles the ABI takes.  There is no CPU path: if
the compiled library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

CODAG_ORC_RLE_V1_I64 = 1
CODAG_ORC_RLE_V2_I64 = 2
CODAG_DEFLATE_RAW = 3
CODAG_ORC_RLE_V1_U64 = 4
CODAG_ORC_RLE_V2_U64 = 5
CODAG_ORC_BYTE_RLE = 6
CODAG_ORC_BOOL_RLE = 7
CODAG_ORC_ZLIB = 8
FORMATS = {"rle_v1": 1, "rle_v2": 2, "deflate": 3, "rle_v1_u64": 4, "rle_v2_u64": 5,
           "byte_rle": 6, "bool_rle": 7, "orc_zlib": 8}

CODAG_OK, CODAG_EINVAL, CODAG_ECUDA, CODAG_ENOMEM, CODAG_ECORRUPT, CODAG_ETIMEOUT = range(6)
CHUNK_STATUS = ["OK", "TRUNCATED", "OUTPUT_OVERFLOW", "OUTPUT_UNDERFLOW", "BAD_HEADER",
                "BAD_HUFFMAN", "BAD_DISTANCE", "BAD_STORED_LEN", "BAD_SPAN", "TIMEOUT"]

_lock = threading.Lock()
_lib = None


class CodagError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """Load libcodag.so (building it first when nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not _build.up_to_date():
            try:
                _build.build()
            except Exception as e:  # no silent fallback: the GPU library is the product
                raise RuntimeError(f"libcodag.so is missing and could not be built: {e}") from e
        L = ctypes.CDLL(_build.LIB_PATH)
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        L.codag_decompress.argtypes = [i32, vp, vp, u64, vp, vp, vp]
        L.codag_decompressed_sizes.argtypes = [i32, vp, vp, u64, vp, vp]
        L.codag_decompress_host.argtypes = [i32, vp, vp, u64, vp, vp, vp, vp, vp, vp]
        L.codag_decompress_batch.argtypes = [vp, vp, vp, u64, vp, vp, vp, vp]
        L.codag_last_chunk_status.argtypes = [vp, u64, vp]
        L.codag_decompress_batch_noalloc.argtypes = [vp, vp, vp, u64, vp, vp, vp, vp]
        L.codag_decompress_batch_ws.argtypes = [vp, vp, vp, u64, vp, vp, vp, vp, u64, vp]
        L.codag_batch_scratch_bytes.argtypes = [u64]
        L.codag_batch_scratch_bytes.restype = u64
        L.codag_batch_graph_create.argtypes = [vp, vp, vp, u64, vp, vp, vp, vp, ctypes.POINTER(vp)]
        L.codag_batch_graph_launch.argtypes = [vp, vp]
        L.codag_batch_graph_destroy.argtypes = [vp]
        L.codag_set_batch_ctas_per_sm.argtypes = [i32]
        L.codag_set_parts_per_chunk.argtypes = [i32]
        L.codag_get_parts_per_chunk.restype = i32
        L.codag_set_input_staging.argtypes = [i32, i32]
        L.codag_set_input_staging.restype = i32
        L.codag_get_input_staging.argtypes = [i32]
        L.codag_get_input_staging.restype = i32
        L.codag_set_deflate_pool_limit.argtypes = [u64]
        L.codag_get_deflate_pool_limit.restype = u64
        ip = ctypes.POINTER(i32)
        L.codag_batch_staging_shapes.argtypes = [ip, ip, i32]
        L.codag_batch_staging_shapes.restype = i32
        L.codag_set_batch_staging.argtypes = [i32, i32]
        L.codag_get_batch_staging.argtypes = [ip, ip]
        L.codag_set_batch_split.argtypes = [i32, i32]
        L.codag_get_batch_split.argtypes = [ip, ip]
        for name in ("codag_set_batch_staging", "codag_get_batch_staging",
                     "codag_set_batch_split", "codag_get_batch_split"):
            getattr(L, name).restype = i32
        L.codag_set_walk_pass.argtypes = [i32, i32]
        L.codag_set_walk_pass.restype = i32
        L.codag_get_walk_pass.argtypes = [i32]
        L.codag_get_walk_pass.restype = i32
        L.codag_set_wait_limit_ns.argtypes = [u64]
        L.codag_get_wait_limit_ns.restype = u64
        for name in ("codag_decompress", "codag_decompressed_sizes", "codag_decompress_batch",
                     "codag_decompress_host",
                     "codag_last_chunk_status", "codag_batch_graph_create",
                     "codag_batch_graph_launch", "codag_batch_graph_destroy",
                     "codag_set_batch_ctas_per_sm", "codag_decompress_batch_noalloc",
                     "codag_set_parts_per_chunk", "codag_decompress_batch_ws"):
            getattr(L, name).restype = i32
        L.codag_get_batch_ctas_per_sm.restype = i32
        L.codag_kernel_launches.restype = ctypes.c_uint64
        L.codag_last_error.restype = ctypes.c_char_p
        L.codag_version.restype = ctypes.c_char_p
        _lib = L
        return L


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch tensor (device or host)
        return x.data_ptr()
    return x.ctypes.data  # numpy array (host)


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st: int, where: str):
    if st != CODAG_OK:
        raise CodagError(st, where, lib().codag_last_error().decode())


def _fmt(f) -> int:
    return FORMATS[f] if isinstance(f, str) else int(f)


def codag_decompress(fmt, comp, comp_offsets, n_chunks: int, out, out_offsets, stream=None):
    """Decode n_chunks chunks of one format (device tensors or raw pointers)."""
    _check(lib().codag_decompress(_fmt(fmt), _ptr(comp), _ptr(comp_offsets), n_chunks, _ptr(out),
                                  _ptr(out_offsets), _stream(stream)), "codag_decompress")


def codag_decompress_host(fmt, h_comp, h_comp_offsets, n_chunks: int, h_out, h_out_offsets,
                          d_comp, d_out, h_status=None, stream=None):
    """Host-to-host decode with the copies overlapped with decoding.  h_*:
    host arrays (numpy, or page-locked torch CPU tensors for overlap);
    d_comp / d_out: device buffers as large as the compressed and decoded
    data.  Asynchronous on `stream`."""
    _check(lib().codag_decompress_host(_fmt(fmt), _ptr(h_comp), _ptr(h_comp_offsets), n_chunks,
                                       _ptr(h_out), _ptr(h_out_offsets), _ptr(d_comp), _ptr(d_out),
                                       _ptr(h_status), _stream(stream)), "codag_decompress_host")


def codag_decompressed_sizes(fmt, comp, comp_offsets, n_chunks: int, sizes_out, stream=None):
    _check(lib().codag_decompressed_sizes(_fmt(fmt), _ptr(comp), _ptr(comp_offsets), n_chunks,
                                          _ptr(sizes_out), _stream(stream)),
           "codag_decompressed_sizes")


def codag_decompress_batch(formats, comp, comp_offsets, n_chunks: int, out, out_offsets,
                           chunk_status=None, stream=None):
    _check(lib().codag_decompress_batch(_ptr(formats), _ptr(comp), _ptr(comp_offsets), n_chunks,
                                        _ptr(out), _ptr(out_offsets), _ptr(chunk_status),
                                        _stream(stream)), "codag_decompress_batch")


def codag_batch_scratch_bytes(n_chunks: int) -> int:
    return lib().codag_batch_scratch_bytes(n_chunks)


def codag_decompress_batch_ws(formats, comp, comp_offsets, n_chunks: int, out, out_offsets,
                              chunk_status, scratch, scratch_bytes: int, stream=None):
    """Batch decode with caller-provided scratch (so batches on several
    streams can run concurrently)."""
    _check(lib().codag_decompress_batch_ws(_ptr(formats), _ptr(comp), _ptr(comp_offsets), n_chunks,
                                           _ptr(out), _ptr(out_offsets), _ptr(chunk_status),
                                           _ptr(scratch), scratch_bytes, _stream(stream)),
           "codag_decompress_batch_ws")


def codag_decompress_batch_noalloc(formats, comp, comp_offsets, n_chunks: int, out, out_offsets,
                                   chunk_status, stream=None):
    """Batch decode that allocates no device memory (scratch is a fixed array
    in the library, at most CODAG_NOALLOC_MAX_CHUNKS chunks per call; calls
    must not overlap on the GPU).  chunk_status is required."""
    _check(lib().codag_decompress_batch_noalloc(_ptr(formats), _ptr(comp), _ptr(comp_offsets),
                                                n_chunks, _ptr(out), _ptr(out_offsets),
                                                _ptr(chunk_status), _stream(stream)),
           "codag_decompress_batch_noalloc")


CODAG_NOALLOC_MAX_CHUNKS = 32768


def codag_last_chunk_status(n: int, stream=None):
    """Per-chunk status of the last plain call as a numpy int32 array."""
    import numpy as np
    host = np.zeros(max(n, 1), dtype=np.int32)
    st = lib().codag_last_chunk_status(host.ctypes.data, n, _stream(stream))
    if st not in (CODAG_OK, CODAG_ECORRUPT):
        _check(st, "codag_last_chunk_status")
    return host[:n]


class BatchGraph:
    """codag_batch_graph_create/launch/destroy as an object."""

    def __init__(self, formats, comp, comp_offsets, n_chunks, out, out_offsets, chunk_status,
                 stream=None):
        h = ctypes.c_void_p()
        _check(lib().codag_batch_graph_create(_ptr(formats), _ptr(comp), _ptr(comp_offsets),
                                              n_chunks, _ptr(out), _ptr(out_offsets),
                                              _ptr(chunk_status), _stream(stream),
                                              ctypes.byref(h)), "codag_batch_graph_create")
        self._h = h

    def launch(self, stream=None):
        _check(lib().codag_batch_graph_launch(self._h, _stream(stream)), "codag_batch_graph_launch")

    def destroy(self):
        if self._h:
            lib().codag_batch_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def codag_batch_graph_create(*args, **kw) -> BatchGraph:
    return BatchGraph(*args, **kw)


def codag_batch_graph_launch(graph: BatchGraph, stream=None):
    graph.launch(stream)


def codag_batch_graph_destroy(graph: BatchGraph):
    graph.destroy()


def codag_set_batch_ctas_per_sm(k: int):
    _check(lib().codag_set_batch_ctas_per_sm(int(k)), "codag_set_batch_ctas_per_sm")


def codag_get_batch_ctas_per_sm() -> int:
    return lib().codag_get_batch_ctas_per_sm()


def codag_set_walk_pass(fmt, mode: int):
    _check(lib().codag_set_walk_pass(_fmt(fmt), int(mode)), "codag_set_walk_pass")


def codag_get_walk_pass(fmt) -> int:
    return lib().codag_get_walk_pass(_fmt(fmt))


def codag_batch_staging_shapes() -> list:
    """Input-ring shapes the batch kernel is compiled for: [(slot_bytes, slots), ...]."""
    n = lib().codag_batch_staging_shapes(None, None, 0)
    a, b = (ctypes.c_int32 * n)(), (ctypes.c_int32 * n)()
    lib().codag_batch_staging_shapes(a, b, n)
    return [(int(a[i]), int(b[i])) for i in range(n)]


def codag_set_batch_staging(slot_bytes: int, slots: int):
    _check(lib().codag_set_batch_staging(int(slot_bytes), int(slots)), "codag_set_batch_staging")


def codag_get_batch_staging() -> tuple:
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().codag_get_batch_staging(ctypes.byref(a), ctypes.byref(b)), "codag_get_batch_staging")
    return int(a.value), int(b.value)


def codag_set_batch_split(split_log2: int, max_parts: int):
    _check(lib().codag_set_batch_split(int(split_log2), int(max_parts)), "codag_set_batch_split")


def codag_get_batch_split() -> tuple:
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().codag_get_batch_split(ctypes.byref(a), ctypes.byref(b)), "codag_get_batch_split")
    return int(a.value), int(b.value)


def codag_set_parts_per_chunk(k: int):
    _check(lib().codag_set_parts_per_chunk(int(k)), "codag_set_parts_per_chunk")


def codag_set_input_staging(fmt, mode: int):
    """0: shared-memory TMA ring, 1: register ring (Deflate, byte / boolean RLE)."""
    _check(lib().codag_set_input_staging(_fmt(fmt), mode), "codag_set_input_staging")


def codag_get_input_staging(fmt) -> int:
    return lib().codag_get_input_staging(_fmt(fmt))


def codag_set_deflate_pool_limit(nbytes: int):
    """Bound on the two-pass Deflate command pool in bytes (0: none)."""
    _check(lib().codag_set_deflate_pool_limit(int(nbytes)), "codag_set_deflate_pool_limit")


def codag_get_deflate_pool_limit() -> int:
    return lib().codag_get_deflate_pool_limit()


def codag_set_wait_limit_ns(ns: int):
    """Bound of device waits on work in progress (default 100 ms; 0: no wait)."""
    _check(lib().codag_set_wait_limit_ns(int(ns)), "codag_set_wait_limit_ns")


def codag_get_wait_limit_ns() -> int:
    return lib().codag_get_wait_limit_ns()


def codag_get_parts_per_chunk() -> int:
    return lib().codag_get_parts_per_chunk()


def codag_kernel_launches() -> int:
    return lib().codag_kernel_launches()


def codag_version() -> str:
    return lib().codag_version().decode()


# short aliases
decompress = codag_decompress
decompressed_sizes = codag_decompressed_sizes
decompress_batch = codag_decompress_batch
last_chunk_status = codag_last_chunk_status
