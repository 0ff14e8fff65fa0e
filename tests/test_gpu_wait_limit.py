"""Bounded device waits, made to run out (codag_set_wait_limit_ns).

Every wait of a decoder on work in progress (a TMA staging copy it needs
next, a segment start another warp of its chunk publishes) is bounded; a
wait that runs out ends the chunk with CHUNK_TIMEOUT after the decoder has
waited, with the default bound, for its own copies in flight.  With the
bound at 0 such waits give up unless already complete: every chunk status
must then be OK or TIMEOUT and nothing else, the device must keep working,
and the next calls at the default bound must be bit-exact again."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2307_03760_gb300 as codag  # noqa: E402
from devutil import assert_parity, run_batch, run_plain, run_sizes  # noqa: E402

TIMEOUT = 9
DEFAULT_NS = 100_000_000


def _cases():
    big = 30000 * 8  # chunks too large to stage: per-warp TMA rings
    return [
        (2, synth.build_chunks([2] * 24, [131072] * 20 + [big, big, 800, 8], seed=51)),
        (1, synth.build_chunks([1] * 12, [65536] * 10 + [big, 16], seed=52)),
        (6, synth.build_chunks([6] * 12, [65536] * 11 + [300000], seed=53)),
        (8, synth.orc_zlib_column(54, total=8 << 20)),
        # a chunk over 128 KiB goes to the persistent one-warp pass after the
        # two Deflate passes, whose ring waits can run out
        (3, synth.build_chunks([3] * 7, [65536] * 6 + [300000], seed=56)),
    ]


def test_zero_wait_bound_gives_timeouts_only_then_exact_again():
    cases = _cases()
    mixed = synth.batched(seed=55, n_chunks=300, lo=512, hi=1 << 19)
    assert codag.codag_get_wait_limit_ns() == DEFAULT_NS
    codag.codag_set_wait_limit_ns(0)
    timeouts = 0
    try:
        for fmt, w in cases:
            _, st = run_plain(fmt, w.comp, w.comp_off, w.out_off)
            assert set(np.unique(st).tolist()) <= {0, TIMEOUT}, (fmt, np.unique(st))
            timeouts += int((st == TIMEOUT).sum())
            if fmt in (1, 2, 3):  # the sizes walks (and the one-warp Deflate sizes) wait too
                _, sst = run_sizes(fmt, w.comp, w.comp_off)
                assert set(np.unique(sst).tolist()) <= {0, TIMEOUT}
        _, bst = run_batch(mixed.formats, mixed.comp, mixed.comp_off, mixed.out_off)
        assert set(np.unique(bst).tolist()) <= {0, TIMEOUT}
        timeouts += int((bst == TIMEOUT).sum())
    finally:
        codag.codag_set_wait_limit_ns(DEFAULT_NS)
    assert timeouts > 0, "no wait ran out: the bound was not applied"
    torch.cuda.synchronize()
    for fmt, w in cases:
        got, st = run_plain(fmt, w.comp, w.comp_off, w.out_off)
        assert (st == 0).all()
        assert_parity(fmt, w.comp, w.comp_off, w.out_off, got, st)
    got, st = run_batch(mixed.formats, mixed.comp, mixed.comp_off, mixed.out_off)
    assert (st == 0).all()
    assert_parity(0, mixed.comp, mixed.comp_off, mixed.out_off, got, st, formats=mixed.formats)
