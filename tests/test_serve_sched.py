"""Serving scheduler on the CPU: arena allocation, admission by memory,
batch chunk tables (checked by decoding them with the oracle) and the
serving loop driven by a fake executor."""
import random

import numpy as np

import oracle
import synth
from paper_2307_03760_gb300.serve import (ALIGN, CODAG_ETIMEOUT, CODAG_OK, Arena, Request,
                                          Scheduler, Server, chunk_table, comp_region)


def _req(rid, w, arrival=0.0):
    return Request(rid, w.formats, w.comp, w.comp_off, w.out_off, arrival)


def test_arena_first_fit_and_coalescing():
    a = Arena(1 << 20)
    rng = random.Random(1)
    live = {}
    for step in range(3000):
        if live and rng.random() < 0.45:
            off = rng.choice(list(live))
            a.free(off)
            del live[off]
        else:
            n = rng.randint(1, 40000)
            off = a.alloc(n)
            if off is not None:
                live[off] = (n + ALIGN - 1) // ALIGN * ALIGN
        spans = sorted(live.items())
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2  # no overlap
        assert a.used == sum(live.values())
    for off in list(live):
        a.free(off)
    assert a.free_list == [(0, 1 << 20)] and a.used == 0


def test_admission_by_memory_and_rejection():
    w = synth.build_chunks([2] * 4, [8192] * 4, 3)
    need = Scheduler.block_bytes(_req(0, w))
    s = Scheduler(budget=need * 2 + ALIGN, max_batch_chunks=1000)
    reqs = [_req(i, w) for i in range(3)]
    for r in reqs:
        assert s.arrive(r)
    s.admit()
    assert [r.rid for r in s.admitted] == [0, 1] and [r.rid for r in s.waiting] == [2]
    big = synth.build_chunks([2], [8 * 100000], 4)
    assert not s.arrive(_req(9, big))  # can never fit the budget
    batch = s.next_batch()
    assert [r.rid for r in batch] == [0, 1]
    s.release(batch[0])
    s.admit()
    assert [r.rid for r in s.admitted] == [2]


def test_chunk_table_decodes_each_request_as_alone():
    """A batch table with gap chunks, decoded by the oracle over one arena,
    gives every request exactly its own output."""
    pool = [synth.build_chunks([f] * n, [s] * n, 10 + i, keep_plain=True)
            for i, (f, n, s) in enumerate([(1, 3, 8192), (3, 2, 5000 // 8 * 8), (2, 5, 16384),
                                           (3, 1, 800), (1, 1, 8)])]
    s = Scheduler(budget=4 << 20, max_batch_chunks=1000)
    reqs = [_req(i, w) for i, w in enumerate(pool)]
    for r in reqs:
        s.arrive(r)
    s.admit()
    s.release(reqs[1])  # leave a hole so the layout has a real gap
    s.admitted = [r for r in s.admitted if r.rid != 1]
    batch = s.next_batch()
    arena = np.zeros(4 << 20, np.uint8)
    for r in batch:
        arena[r.comp_at:r.comp_at + r.comp_bytes] = r.comp
    fm, co, oo, index = chunk_table(batch)
    assert (np.diff(co.astype(np.int64)) >= 0).all() and (np.diff(oo.astype(np.int64)) >= 0).all()
    out, st = oracle.decode(0, arena, co, oo, formats=fm)
    for r, i in zip(batch, index):
        assert (st[i:i + r.n] == 0).all()
        got = out[int(oo[i]):int(oo[i]) + r.out_bytes]
        assert np.array_equal(got, pool[r.rid].plain)
    gaps = np.nonzero(fm == 0)[0]
    assert len(gaps) == len(batch) - 1 and (st[gaps] == oracle.BAD_HEADER).all()


class FakeExecutor:
    """Completes each batch after `delay` seconds of fake time; decodes with
    the oracle so results can be checked."""

    def __init__(self, budget, streams, clock, delay=0.002):
        self.arena = np.zeros(budget, np.uint8)
        self.slots = [{"busy": None} for _ in range(streams)]
        self.clock, self.delay = clock, delay
        self.launched = []

    def free_slot(self):
        return next((s for s in self.slots if s["busy"] is None), None)

    def launch(self, slot, batch, inputs):
        for r in batch:
            self.arena[r.comp_at:r.comp_at + r.comp_bytes] = inputs[r.rid]
        fm, co, oo, index = chunk_table(batch)
        out, st = oracle.decode(0, self.arena, co, oo, formats=fm)
        for r, i in zip(batch, index):
            self.arena[r.out_at:r.out_at + r.out_bytes] = out[int(oo[i]):int(oo[i]) + r.out_bytes]
        slot.update(busy=batch, t=self.clock() + self.delay, st=[st[i:i + r.n] for r, i in zip(batch, index)])
        self.launched.append([r.rid for r in batch])

    def poll(self):
        done = []
        for s in self.slots:
            if s["busy"] is not None and self.clock() >= s["t"]:
                done.append((s["busy"], s["st"]))
                s["busy"] = None
        return done

    def read_output(self, r):
        return self.arena[r.out_at:r.out_at + r.out_bytes].copy()


def test_serving_loop_continuous_batching_with_fake_executor():
    pool = [synth.build_chunks([f] * 2, [4096] * 2, 20 + f, keep_plain=True) for f in (1, 2, 3)]
    t = [0.0]
    clock = lambda: t[0]  # noqa: E731
    reqs = [Request(i, pool[i % 3].formats, pool[i % 3].comp, pool[i % 3].comp_off,
                    pool[i % 3].out_off, arrival=0.001 * i) for i in range(30)]
    inputs = {r.rid: r.comp for r in reqs}
    ex = FakeExecutor(budget=1 << 20, streams=2, clock=clock)

    def tick():
        t[0] += 0.0005
        return t[0]

    srv = Server(budget=1 << 20, streams=2, executor=ex, clock=tick, keep_results=True)
    stats = srv.run(reqs, inputs, time_limit=10.0)
    assert stats.completed == 30 and stats.rejected == 0
    assert stats.status == CODAG_OK and stats.timed_out == 0
    assert any(len(b) > 1 for b in ex.launched)  # arrivals during a batch were batched together
    for r in reqs:
        assert (r.status == 0).all()
        assert np.array_equal(r.result, pool[r.rid % 3].plain)
        assert r.t_done >= r.arrival


def test_serving_loop_deadline_returns_etimeout():
    """Batches that never complete: the loop stops polling at its deadline,
    reports CODAG_ETIMEOUT and marks exactly the unfinished requests."""
    pool = [synth.build_chunks([2] * 2, [4096] * 2, 30, keep_plain=True)]
    t = [0.0]

    def tick():
        t[0] += 0.001
        return t[0]

    ex = FakeExecutor(budget=1 << 20, streams=2, clock=tick, delay=0.004)
    reqs = [Request(i, pool[0].formats, pool[0].comp, pool[0].comp_off, pool[0].out_off,
                    arrival=0.0005 * i) for i in range(20)]
    inputs = {r.rid: r.comp for r in reqs}
    slow = ex.poll

    def poll():  # batches launched after the first two never finish
        return [d for d in slow() if min(r.rid for r in d[0]) < 2]

    ex.poll = poll
    srv = Server(budget=1 << 20, streams=2, executor=ex, clock=tick)
    stats = srv.run(reqs, inputs, time_limit=0.2)
    assert stats.status == CODAG_ETIMEOUT
    assert stats.completed >= 1 and stats.timed_out == 20 - stats.completed
    assert all(r.timed_out == (r.t_done < 0) for r in reqs)
    assert stats.summary()["status"] == "ETIMEOUT"
