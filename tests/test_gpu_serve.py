"""Serving on the GPU: requests that arrive while others run are batched
into the persistent kernel on several streams; every request's output must
be bit-identical to the same request decoded alone (and to its input
column)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2307_03760_gb300 as codag  # noqa: E402
from devutil import run_batch  # noqa: E402
from paper_2307_03760_gb300.serve import Request, Server  # noqa: E402


def test_requests_same_alone_and_in_the_mix():
    pool = synth.serving_pool(seed=3, n_payloads=9, lo=64 * 1024, hi=2 << 20, keep_plain=True)
    times, pick = synth.poisson_arrivals(3, rate=4000.0, duration=0.03, n_payloads=len(pool))
    reqs = [Request(i, pool[p].formats, pool[p].comp, pool[p].comp_off, pool[p].out_off,
                    arrival=float(t)) for i, (t, p) in enumerate(zip(times, pick))]
    assert len(reqs) >= 40
    inputs = {r.rid: torch.from_numpy(r.comp).pin_memory() for r in reqs}
    srv = Server(budget=256 << 20, streams=3, max_batch_chunks=8192, keep_results=True)
    stats = srv.run(reqs, inputs, time_limit=30.0)
    assert stats.completed == len(reqs) and stats.rejected == 0
    assert stats.batches < len(reqs)  # arrivals were batched together
    alone = {}
    for p, w in enumerate(pool):
        out, st = run_batch(w.formats, w.comp, w.comp_off, w.out_off)
        assert (st == 0).all()
        alone[p] = out
    for r, p in zip(reqs, pick):
        assert (r.status == 0).all()
        assert np.array_equal(r.result, alone[p])      # same as decoded alone
        assert np.array_equal(r.result, pool[p].plain)  # and the original column


def test_oversized_request_is_rejected_not_run():
    w = synth.build_chunks([2], [8 << 20], 5)
    small = synth.build_chunks([3], [4096], 6)
    reqs = [Request(0, w.formats, w.comp, w.comp_off, w.out_off, 0.0),
            Request(1, small.formats, small.comp, small.comp_off, small.out_off, 0.0)]
    inputs = {r.rid: torch.from_numpy(r.comp).pin_memory() for r in reqs}
    srv = Server(budget=1 << 20, streams=1, max_batch_chunks=64, keep_results=True)
    stats = srv.run(reqs, inputs, time_limit=10.0)
    assert stats.rejected == 1 and stats.completed == 1 and reqs[0].rejected
    assert (reqs[1].status == 0).all()
