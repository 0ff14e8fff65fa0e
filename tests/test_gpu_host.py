"""codag_decompress_host: host buffers in, host buffers out, with the copies
of one slice overlapping the decode of the next.  Bit-exact against the
oracle, per-chunk statuses included, over several slices, corrupted and
empty chunks, back-to-back calls and a non-default stream."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2307_03760_gb300 as codag  # noqa: E402

THREADS = os.cpu_count() or 4
DEV = torch.device("cuda:0")


def _pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.empty(max(a.size, 16), dtype=torch.uint8).pin_memory()
    t[: a.size] = torch.from_numpy(np.ascontiguousarray(a))
    return t


def _run_host(w, comp=None, stream=None):
    comp = w.comp if comp is None else comp
    fmt = int(w.formats[0])
    h_comp = _pinned(comp)
    h_out = torch.full((max(w.out_bytes, 16),), 0xA5, dtype=torch.uint8).pin_memory()
    h_st = torch.full((w.n,), -1, dtype=torch.int32).pin_memory()
    d_comp = torch.empty(max(w.comp_bytes, 16), dtype=torch.uint8, device=DEV)
    d_out = torch.empty(max(w.out_bytes, 16), dtype=torch.uint8, device=DEV)
    codag.codag_decompress_host(fmt, h_comp, w.comp_off, w.n, h_out, w.out_off, d_comp, d_out,
                                h_st, stream=stream)
    (stream or torch.cuda.current_stream()).synchronize()
    return h_out[: w.out_bytes].numpy().copy(), h_st.numpy().copy()


def _check(w, got, st, comp=None):
    comp = w.comp if comp is None else comp
    exp, est = oracle.decode(int(w.formats[0]), comp, w.comp_off, w.out_off, threads=THREADS)
    assert np.array_equal(st, est[: w.n])
    for c in np.nonzero(est[: w.n] == 0)[0]:
        a, b = int(w.out_off[c]), int(w.out_off[c + 1])
        assert np.array_equal(got[a:b], exp[a:b]), f"chunk {c} differs"
    return est


@pytest.mark.parametrize("name,total,chunk", [("rle_v1", 8 * synth.MiB, 65536),
                                              ("rle_v2", 72 * synth.MiB, 8192),
                                              ("deflate", 40 * synth.MiB, 4096),
                                              ("byte_rle", 40 * synth.MiB, 10240)])
def test_host_columns(name, total, chunk):
    """Small chunks, so that the columns are cut into several slices (one for
    the 8 MiB RLE v1 column)."""
    w = {"rle_v1": synth.rle_v1_column, "rle_v2": synth.rle_v2_column,
         "deflate": synth.deflate_column, "byte_rle": synth.byte_rle_column}[name](
        seed=5, total=total, chunk=chunk)
    got, st = _run_host(w)
    assert (st == 0).all()
    _check(w, got, st)


def test_host_errors_and_empty_chunks():
    """Chunks whose output span is 8 bytes short or long report
    OUTPUT_OVERFLOW / OUTPUT_UNDERFLOW; a flipped header byte gives whatever
    the oracle says; empty chunks decode to nothing; the rest are exact."""
    fmts, sizes = [], []
    rng = np.random.default_rng(7)
    for i in range(3000):
        fmts.append(synth.RLE_V2_I64)
        sizes.append(0 if i % 37 == 5 else int(rng.integers(1, 6)) * 8192)
    w = synth.build_chunks(fmts, sizes, 11, name="mixed_sizes")
    spans = np.diff(w.out_off).astype(np.int64)
    for c in range(3, w.n, 23):
        spans[c] += -8 if spans[c] >= 8 else 8
    for c in range(7, w.n, 29):
        spans[c] += 8
    out_off = np.zeros(w.n + 1, np.uint64)
    out_off[1:] = np.cumsum(spans)
    comp = w.comp.copy()
    for c in range(11, w.n, 31):
        a, b = int(w.comp_off[c]), int(w.comp_off[c + 1])
        if b > a:
            comp[a] ^= 0xC0  # another sub-encoding for the first run
    w2 = synth.Chunked(comp, w.comp_off, out_off, w.formats, None, "mixed_sizes_bad")
    got, st = _run_host(w2)
    est = _check(w2, got, st)
    assert (est == 2).any() and (est == 3).any() and (est == 0).any()


def test_host_back_to_back_and_side_stream():
    w1 = synth.rle_v2_column(seed=8, total=40 * synth.MiB, chunk=8192)
    w2 = synth.deflate_column(seed=9, total=20 * synth.MiB, chunk=4096)
    s = torch.cuda.Stream()
    for w in (w1, w2, w1):
        got, st = _run_host(w, stream=s)
        assert (st == 0).all()
        _check(w, got, st)
    # statuses of the last call also stay in the workspace
    assert (codag.codag_last_chunk_status(w1.n) == 0).all()
