"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; argument checks that need no GPU return EINVAL."""
import ctypes
import glob
import os
import re

import pytest

import paper_2307_03760_gb300 as codag

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(codag_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("codag_decompress", "codag_decompressed_sizes", "codag_decompress_batch",
                     "codag_last_chunk_status"):
        assert required in names


@pytest.mark.parametrize("name", declared_functions())
def test_library_exports(name):
    L = codag.lib()
    assert hasattr(L, name), f"{name} declared in include/ but not exported"


def test_library_is_in_tree():
    assert os.path.realpath(codag.library_path()).startswith(os.path.realpath(ROOT))


def test_version():
    assert codag.codag_version().startswith("codag-gb300")


def test_argument_errors_without_gpu():
    L = codag.lib()
    # unknown format, checked before any CUDA call
    assert L.codag_decompress(42, None, None, 0, None, None, None) == codag.CODAG_EINVAL
    # zero chunks is a no-op
    assert L.codag_decompress(1, None, None, 0, None, None, None) == codag.CODAG_OK
    # NULL comp with chunks
    assert L.codag_decompress(1, None, None, 5, None, None, None) == codag.CODAG_EINVAL
    # misaligned comp pointer (never dereferenced)
    assert L.codag_decompress(3, 0x1001, 0x2000, 5, 0x3000, 0x4000, None) == codag.CODAG_EINVAL
    # misaligned RLE output
    assert L.codag_decompress(1, 0x1000, 0x2000, 5, 0x3004, 0x4000, None) == codag.CODAG_EINVAL
    assert L.codag_decompressed_sizes(2, 0x1000, 0x2000, 5, None, None) == codag.CODAG_EINVAL
    assert L.codag_decompress_batch(None, 0x1000, 0x2000, 5, 0x3000, 0x4000, None, None) == codag.CODAG_EINVAL
    assert L.codag_set_batch_ctas_per_sm(-1) == codag.CODAG_EINVAL
    assert b"aligned" in L.codag_last_error() or b"NULL" in L.codag_last_error() or L.codag_last_error()
    assert L.codag_batch_graph_launch(None, None) == codag.CODAG_EINVAL


def test_host_entry_argument_errors_without_gpu():
    import numpy as np
    L = codag.lib()
    h = np.zeros(64, np.uint8)
    off = np.array([0, 8, 16], np.uint64)
    dec = np.array([0, 16, 8], np.uint64)  # decreasing
    P = lambda a: a.ctypes.data
    # unknown format, zero chunks
    assert L.codag_decompress_host(42, P(h), P(off), 2, P(h), P(off), 0x1000, 0x2000, None, None) == codag.CODAG_EINVAL
    assert L.codag_decompress_host(1, None, None, 0, None, None, None, None, None, None) == codag.CODAG_OK
    # NULL host or device buffers
    assert L.codag_decompress_host(1, None, P(off), 2, P(h), P(off), 0x1000, 0x2000, None, None) == codag.CODAG_EINVAL
    assert L.codag_decompress_host(1, P(h), P(off), 2, P(h), P(off), None, 0x2000, None, None) == codag.CODAG_EINVAL
    # misaligned device buffers (never dereferenced)
    assert L.codag_decompress_host(3, P(h), P(off), 2, P(h), P(off), 0x1008, 0x2000, None, None) == codag.CODAG_EINVAL
    assert L.codag_decompress_host(2, P(h), P(off), 2, P(h), P(off), 0x1000, 0x2004, None, None) == codag.CODAG_EINVAL
    # decreasing offsets, compressed or decoded
    assert L.codag_decompress_host(2, P(h), P(dec), 2, P(h), P(off), 0x1000, 0x2000, None, None) == codag.CODAG_EINVAL
    assert L.codag_decompress_host(2, P(h), P(off), 2, P(h), P(dec), 0x1000, 0x2000, None, None) == codag.CODAG_EINVAL
    assert b"non-decreasing" in L.codag_last_error()


def test_input_staging_setting():
    L = codag.lib()
    assert L.codag_set_input_staging(1, 1) == codag.CODAG_EINVAL  # RLE v1 always stages in smem
    assert L.codag_set_input_staging(3, 2) == codag.CODAG_EINVAL
    assert L.codag_get_input_staging(2) == -1
    for f in (3, 6, 7):
        assert L.codag_set_input_staging(f, 1) == codag.CODAG_OK
        assert L.codag_get_input_staging(f) == 1
        assert L.codag_set_input_staging(f, 0) == codag.CODAG_OK
        assert L.codag_get_input_staging(f) == 0


def test_batch_staging_selection():
    """The batch kernel's compiled ring shapes are listed, each can be
    selected, anything else is refused and leaves the selection alone."""
    shapes = codag.codag_batch_staging_shapes()
    assert shapes == [(256, 8), (512, 8), (1024, 4), (2048, 4)]
    assert codag.codag_get_batch_staging() == (1024, 4)  # default
    L = codag.lib()
    try:
        for shape in shapes:
            codag.codag_set_batch_staging(*shape)
            assert codag.codag_get_batch_staging() == shape
        codag.codag_set_batch_staging(512, 8)
        for bad in ((512, 4), (1024, 3), (4096, 4), (-1, 4), (0, 4)):
            assert L.codag_set_batch_staging(*bad) == codag.CODAG_EINVAL
            assert codag.codag_get_batch_staging() == (512, 8)
        assert b"no batch kernel is compiled" in L.codag_last_error()
        # a short array takes only the first shapes; the count is still returned
        a = (ctypes.c_int32 * 2)()
        assert L.codag_batch_staging_shapes(a, None, 2) == len(shapes)
        assert list(a) == [256, 512]
        codag.codag_set_batch_staging(0, 0)
        assert codag.codag_get_batch_staging() == (1024, 4)
    finally:
        codag.codag_set_batch_staging(0, 0)


def test_batch_split_selection():
    assert codag.codag_get_batch_split() == (16, 16)  # default
    L = codag.lib()
    try:
        codag.codag_set_batch_split(12, 32)
        assert codag.codag_get_batch_split() == (12, 32)
        codag.codag_set_batch_split(20, 1)
        assert codag.codag_get_batch_split() == (20, 1)
        for bad in ((7, 4), (41, 4), (16, 0), (16, 33), (0, 4), (16, -1)):
            assert L.codag_set_batch_split(*bad) == codag.CODAG_EINVAL
            assert codag.codag_get_batch_split() == (20, 1)
        assert L.codag_get_batch_split(None, None) == codag.CODAG_EINVAL
        codag.codag_set_batch_split(0, 0)
        assert codag.codag_get_batch_split() == (16, 16)
    finally:
        codag.codag_set_batch_split(0, 0)


def test_walk_pass_setting():
    L = codag.lib()
    assert codag.codag_get_walk_pass(2) == 0 and codag.codag_get_walk_pass(5) == 0  # default
    assert codag.codag_get_walk_pass(1) == -1 and codag.codag_get_walk_pass(3) == -1
    assert L.codag_set_walk_pass(1, 0) == codag.CODAG_EINVAL
    assert L.codag_set_walk_pass(2, 2) == codag.CODAG_EINVAL
    try:
        codag.codag_set_walk_pass(5, 1)
        assert codag.codag_get_walk_pass(2) == 1
    finally:
        codag.codag_set_walk_pass(2, 0)
    assert codag.codag_get_walk_pass(2) == 0


def test_deflate_pool_limit_setting():
    assert codag.codag_get_deflate_pool_limit() == 0  # default: no bound
    codag.codag_set_deflate_pool_limit(1 << 20)
    assert codag.codag_get_deflate_pool_limit() == 1 << 20
    codag.codag_set_deflate_pool_limit(0)
    assert codag.codag_get_deflate_pool_limit() == 0


def test_wait_limit_default():
    assert codag.codag_get_wait_limit_ns() == 100_000_000


def test_python_binding_names_match_abi():
    for name in declared_functions():
        if name in ("codag_last_error",):
            continue
        assert hasattr(codag, name), f"binding lacks {name}"
