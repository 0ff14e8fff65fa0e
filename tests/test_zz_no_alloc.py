"""The allocation-free batch entry point, through the C ABI.

codag_decompress_batch_noalloc serves callers that cannot let the library
allocate device memory (their own memory budget or pool, or loops that
cannot take a first-call cudaMalloc).  Its output and per-chunk status must
equal those of codag_decompress_batch bit for bit, on two calls in a row
that share the library's fixed scratch array.  This file is collected last
so that a run stopping at the first failure has run every other test."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2307_03760_gb300 as codag  # noqa: E402
from devutil import DEV, dev_u8, dev_u64  # noqa: E402


def _upload(w):
    return (dev_u8(w.formats), dev_u8(w.comp), dev_u64(w.comp_off), dev_u64(w.out_off))


def _reference(w):
    fm, comp, coff, ooff = _upload(w)
    out = torch.zeros(w.out_bytes + 16, dtype=torch.uint8, device=DEV)
    st = torch.full((w.n,), -1, dtype=torch.int32, device=DEV)
    codag.codag_decompress_batch(fm, comp, coff, w.n, out, ooff, st)
    torch.cuda.synchronize()
    return out[: w.out_bytes].cpu().numpy(), st.cpu().numpy()


def _noalloc(w):
    fm, comp, coff, ooff = _upload(w)
    out = torch.full((w.out_bytes + 16,), 0x5A, dtype=torch.uint8, device=DEV)
    st = torch.full((w.n,), -1, dtype=torch.int32, device=DEV)
    codag.codag_decompress_batch_noalloc(fm, comp, coff, w.n, out, ooff, st)
    torch.cuda.synchronize()
    return out[: w.out_bytes].cpu().numpy(), st.cpu().numpy()


def test_noalloc_matches_batch_two_calls_in_a_row():
    first = synth.batched(seed=17, n_chunks=3000, lo=512, hi=1 << 17, keep_plain=True)
    second = synth.batched(seed=18, n_chunks=1200, lo=512, hi=1 << 16, keep_plain=True)
    for w in (first, second):  # the second call reuses the scratch the first left behind
        ref_out, ref_st = _reference(w)
        out, st = _noalloc(w)
        assert (ref_st == 0).all()
        assert np.array_equal(st, ref_st)
        assert np.array_equal(out, ref_out)
        assert np.array_equal(out, w.plain)


def test_noalloc_follows_staging_and_split_choice():
    """The no-alloc entry point launches the selected ring shape and split rule."""
    w = synth.batched(seed=21, n_chunks=400, lo=512, hi=1 << 19, keep_plain=True)
    try:
        for shape, split in (((256, 8), (12, 32)), ((2048, 4), (16, 1))):
            codag.codag_set_batch_staging(*shape)
            codag.codag_set_batch_split(*split)
            out, st = _noalloc(w)
            assert (st == 0).all(), shape
            assert np.array_equal(out, w.plain), shape
    finally:
        codag.codag_set_batch_staging(0, 0)
        codag.codag_set_batch_split(0, 0)


def test_noalloc_rejects_too_many_chunks():
    n = codag.CODAG_NOALLOC_MAX_CHUNKS + 1
    dummy = torch.zeros(64, dtype=torch.uint8, device=DEV)
    with pytest.raises(codag.CodagError) as e:
        codag.codag_decompress_batch_noalloc(dummy, dummy, dummy, n, dummy, dummy, dummy)
    assert e.value.status == codag.CODAG_EINVAL
    assert "exceeds the maximum" in str(e.value)


FIRST_CALL_SCRIPT = r"""
import sys
sys.path[:0] = [ROOT, TESTS]
import numpy as np
import torch
import synth
import paper_2307_03760_gb300 as codag
from devutil import DEV, dev_u8, dev_u64
torch.cuda.set_device(DEV)
w = synth.batched(seed=19, n_chunks=700, lo=512, hi=1 << 18, keep_plain=True)
args = (dev_u8(w.formats), dev_u8(w.comp), dev_u64(w.comp_off), w.n)
ooff = dev_u64(w.out_off)
out = torch.full((w.out_bytes + 16,), 0x5A, dtype=torch.uint8, device=DEV)
st = torch.full((w.n,), -1, dtype=torch.int32, device=DEV)
# the first call of any entry point in this process: the no-allocation
# entry point's own per-device set-up runs here, with no workspace created
codag.codag_decompress_batch_noalloc(*args, out, ooff, st)
torch.cuda.synchronize()
assert (st.cpu().numpy() == 0).all(), "noalloc statuses"
assert np.array_equal(out[: w.out_bytes].cpu().numpy(), w.plain), "noalloc bytes"
ref = torch.zeros_like(out)
rst = torch.full_like(st, -1)
codag.codag_decompress_batch(*args, ref, ooff, rst)
torch.cuda.synchronize()
assert (rst.cpu().numpy() == 0).all()
assert np.array_equal(ref[: w.out_bytes].cpu().numpy(), w.plain)
print("first-call ok")
"""


def test_noalloc_first_call_in_a_fresh_process():
    """The entry point works as the very first library call of a process, so
    its own set-up (scratch address, kernel attribute, occupancy) is what is
    exercised, not state left behind by the ordinary entry points."""
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    script = FIRST_CALL_SCRIPT.replace("ROOT", repr(root)).replace("TESTS", repr(here))
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "first-call ok" in r.stdout
