"""Full-size workloads on the GPU, bit-exact against the oracle on every
chunk (the oracle runs chunk ranges on all host cores)."""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from devutil import assert_parity, run_batch, run_plain  # noqa: E402

THREADS = os.cpu_count() or 4


@pytest.mark.parametrize("name", ["rle_v1", "rle_v2", "deflate"])
def test_full_column(name):
    """In the launch configuration the benchmark times: the committed
    autotuner table applied for this family."""
    import paper_2307_03760_gb300 as codag
    from paper_2307_03760_gb300 import autotune
    w = {"rle_v1": synth.rle_v1_column, "rle_v2": synth.rle_v2_column,
         "deflate": synth.deflate_column}[name](seed=1)
    fmt = int(w.formats[0])
    autotune.apply(n_chunks=None, family=name)
    try:
        got, st = run_plain(fmt, w.comp, w.comp_off, w.out_off)
        if name == "deflate":
            # the first call may leave chunks past the Deflate command pool to
            # the one-warp decoder (the pool then grows to this call's need);
            # the benchmark times later calls, where the two passes take all
            assert (st == 0).all()
            assert_parity(fmt, w.comp, w.comp_off, w.out_off, got, st, threads=THREADS)
            got, st = run_plain(fmt, w.comp, w.comp_off, w.out_off)
    finally:
        codag.codag_set_parts_per_chunk(0)
        codag.codag_set_batch_ctas_per_sm(0)
        for f in (3, 6, 7):
            codag.codag_set_input_staging(f, 0)
    assert (st == 0).all()
    assert_parity(fmt, w.comp, w.comp_off, w.out_off, got, st, threads=THREADS)


def test_full_batched():
    w = synth.batched(seed=1)
    got, st = run_batch(w.formats, w.comp, w.comp_off, w.out_off)
    assert (st == 0).all()
    assert_parity(0, w.comp, w.comp_off, w.out_off, got, st, formats=w.formats, threads=THREADS)
