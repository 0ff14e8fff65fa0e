"""Continuous-batching decompression server on one GPU.

Requests (each: a list of compressed chunks of any supported format, with
the decoded size of each chunk) arrive over time.  The server keeps every
buffer device-resident: an input arena for compressed bytes and an output
arena for decoded bytes, both carved from a fixed HBM budget.  A request is
admitted when both arenas have room for it; admitted requests that are not
yet on the GPU are packed into one batch (one chunk table) and launched with
``codag_decompress_batch_ws`` on a free stream, while earlier batches may
still be running on other streams, so new work overlaps in-flight work.  When
a batch's event completes its requests are done: latency is arrival ->
completion seen by the host; the arena space is freed for new admissions.

The decoding itself is the library's persistent batch kernel; this module is
host-side scheduling only (admission, batching, completion), written so the
scheduling logic can be driven on the CPU with a fake executor in tests.
"""
from __future__ import annotations

import bisect
import time
from dataclasses import dataclass, field

import numpy as np

ALIGN = 256
# the library's call statuses that the serving loop reports (include/codag.h)
CODAG_OK = 0
CODAG_ETIMEOUT = 5


class Arena:
    """First-fit allocator over [0, size) with coalescing free list."""

    def __init__(self, size: int):
        self.size = size
        self.free_list = [(0, size)]  # sorted (offset, length)
        self.used = 0
        self.live = {}

    def alloc(self, nbytes: int) -> int | None:
        n = max(ALIGN, (nbytes + ALIGN - 1) // ALIGN * ALIGN)
        for i, (off, ln) in enumerate(self.free_list):
            if ln >= n:
                if ln == n:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + n, ln - n)
                self.live[off] = n
                self.used += n
                return off
        return None

    def free(self, off: int):
        n = self.live.pop(off)
        self.used -= n
        i = bisect.bisect_left(self.free_list, (off, 0))
        self.free_list.insert(i, (off, n))
        # coalesce with neighbours
        if i + 1 < len(self.free_list) and off + n == self.free_list[i + 1][0]:
            self.free_list[i] = (off, n + self.free_list[i + 1][1])
            self.free_list.pop(i + 1)
        if i > 0 and self.free_list[i - 1][0] + self.free_list[i - 1][1] == off:
            po, pn = self.free_list[i - 1]
            self.free_list[i - 1] = (po, pn + self.free_list[i][1])
            self.free_list.pop(i)

    def fits(self, nbytes: int) -> bool:
        n = max(ALIGN, (nbytes + ALIGN - 1) // ALIGN * ALIGN)
        return any(ln >= n for _, ln in self.free_list)


@dataclass
class Request:
    rid: int
    formats: np.ndarray    # uint8 per chunk
    comp: np.ndarray       # uint8, concatenated compressed chunks (host)
    comp_off: np.ndarray   # uint64[n+1], local
    out_off: np.ndarray    # uint64[n+1], local (RLE chunk sizes multiples of 8)
    arrival: float = 0.0
    comp_at: int = -1
    out_at: int = -1
    t_launch: float = -1.0
    t_done: float = -1.0
    status: np.ndarray | None = None
    rejected: bool = False
    timed_out: bool = False  # not completed when the loop's deadline passed
    result: np.ndarray | None = None

    @property
    def n(self) -> int:
        return len(self.comp_off) - 1

    @property
    def comp_bytes(self) -> int:
        return int(self.comp_off[-1])

    @property
    def out_bytes(self) -> int:
        return int(self.out_off[-1])


class Scheduler:
    """Admission and batching policy, independent of the device.

    One arena holds every admitted request as a block [compressed | decoded]
    so that, with requests ordered by block offset, both the compressed and
    the decoded offsets of a batch's chunk table increase; the space between
    two requests becomes a gap chunk (format 0, which the library marks
    BAD_HEADER without reading or writing anything)."""

    def __init__(self, budget: int, max_batch_chunks: int):
        self.arena = Arena(budget)
        self.max_batch_chunks = max_batch_chunks
        self.waiting: list[Request] = []   # arrived, not admitted
        self.admitted: list[Request] = []  # memory reserved, not launched

    @staticmethod
    def block_bytes(r: Request) -> int:
        return comp_region(r) + r.out_bytes

    def arrive(self, r: Request) -> bool:
        """Queue a request; reject it outright if it can never fit."""
        if self.block_bytes(r) + ALIGN > self.arena.size or 2 * r.n + 1 > self.max_batch_chunks:
            r.rejected = True
            return False
        self.waiting.append(r)
        return True

    def admit(self):
        """Admit waiting requests in arrival order while memory allows."""
        while self.waiting:
            r = self.waiting[0]
            b = self.arena.alloc(self.block_bytes(r))
            if b is None:
                break
            r.comp_at, r.out_at = b, b + comp_region(r)
            self.admitted.append(self.waiting.pop(0))

    def next_batch(self) -> list[Request]:
        batch, chunks = [], 0
        while self.admitted and chunks + self.admitted[0].n + 1 <= self.max_batch_chunks:
            r = self.admitted.pop(0)
            batch.append(r)
            chunks += r.n + 1
        return batch

    def release(self, r: Request):
        self.arena.free(r.comp_at)


def comp_region(r: Request) -> int:
    """Bytes reserved for a request's compressed input (room for the decoder's
    16-byte-rounded reads past its last chunk)."""
    return (r.comp_bytes + 64 + ALIGN - 1) // ALIGN * ALIGN


def chunk_table(batch: list[Request]):
    """(formats, comp_off, out_off, index) of a batch, offsets from the arena
    base.  Requests are laid out in block order with a gap chunk (format 0)
    after each; index[i] = position in the table of request i's first chunk."""
    order = sorted(range(len(batch)), key=lambda i: batch[i].comp_at)
    fm, co, oo = [], [], []
    index = [0] * len(batch)
    pos = 0
    for i in order:
        r = batch[i]
        index[i] = pos
        fm.append(r.formats.astype(np.uint8))
        co.append(r.comp_off[:-1] + np.uint64(r.comp_at))
        oo.append(r.out_off[:-1] + np.uint64(r.out_at))
        # gap chunk: from this request's ends to the next request's starts
        fm.append(np.zeros(1, np.uint8))
        co.append(np.array([r.comp_at + r.comp_bytes], np.uint64))
        oo.append(np.array([r.out_at + r.out_bytes], np.uint64))
        pos += r.n + 1
    last = batch[order[-1]]
    fm = np.concatenate(fm)[:-1]  # the final gap chunk is not needed
    co = np.concatenate(co)
    oo = np.concatenate(oo)
    co[-1] = last.comp_at + last.comp_bytes
    oo[-1] = last.out_at + last.out_bytes
    return fm, co, oo, index


@dataclass
class Stats:
    latencies: list = field(default_factory=list)
    bytes_done: int = 0
    completed: int = 0
    rejected: int = 0
    batches: int = 0
    timed_out: int = 0
    status: int = CODAG_OK  # CODAG_ETIMEOUT when requests were left at the deadline
    wall: float = 0.0

    def summary(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"completed": self.completed, "rejected": self.rejected, "batches": self.batches,
                "timed_out": self.timed_out, "status": "ETIMEOUT" if self.status else "OK",
                "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                "mean_ms": round(float(lat.mean()) * 1e3, 3),
                "GBps": round(self.bytes_done / max(self.wall, 1e-9) / 1e9, 2),
                "wall_s": round(self.wall, 3)}


class GpuExecutor:
    """Runs batches with codag_decompress_batch_ws on a pool of streams; all
    buffers (arena, chunk tables, scratch) are allocated once up front."""

    def __init__(self, budget: int, streams: int = 4, max_batch_chunks: int = 32768,
                 device: int = 0):
        import torch

        import paper_2307_03760_gb300 as codag
        self.torch, self.codag = torch, codag
        self.dev = torch.device("cuda", device)
        self.arena = torch.empty(budget, dtype=torch.uint8, device=self.dev)
        self.max_chunks = max_batch_chunks
        sb = codag.codag_batch_scratch_bytes(max_batch_chunks)
        self.scratch_bytes = sb
        self.slots = []
        for _ in range(streams):
            self.slots.append({
                "stream": torch.cuda.Stream(self.dev),
                "scratch": torch.empty(sb, dtype=torch.uint8, device=self.dev),
                "fm": torch.empty(max_batch_chunks, dtype=torch.uint8, device=self.dev),
                "co": torch.empty(max_batch_chunks + 1, dtype=torch.int64, device=self.dev),
                "oo": torch.empty(max_batch_chunks + 1, dtype=torch.int64, device=self.dev),
                "status": torch.empty(max_batch_chunks, dtype=torch.int32, device=self.dev),
                "h_fm": torch.empty(max_batch_chunks, dtype=torch.uint8).pin_memory(),
                "h_co": torch.empty(max_batch_chunks + 1, dtype=torch.int64).pin_memory(),
                "h_oo": torch.empty(max_batch_chunks + 1, dtype=torch.int64).pin_memory(),
                "busy": None, "event": None,
            })

    def free_slot(self):
        for s in self.slots:
            if s["busy"] is None:
                return s
        return None

    def launch(self, slot, batch: list[Request], pinned_inputs: dict):
        torch, codag = self.torch, self.codag
        stream = slot["stream"]
        fm, co, oo, index = chunk_table(batch)
        n = len(fm)
        slot["h_fm"].numpy()[:n] = fm
        slot["h_co"].numpy().view(np.uint64)[: n + 1] = co
        slot["h_oo"].numpy().view(np.uint64)[: n + 1] = oo
        with torch.cuda.stream(stream):
            # the slot's host staging is reused only after this batch completes
            for r in batch:
                if r.comp_bytes:
                    self.arena[r.comp_at:r.comp_at + r.comp_bytes].copy_(
                        pinned_inputs[r.rid][:r.comp_bytes], non_blocking=True)
            slot["fm"][:n].copy_(slot["h_fm"][:n], non_blocking=True)
            slot["co"][: n + 1].copy_(slot["h_co"][: n + 1], non_blocking=True)
            slot["oo"][: n + 1].copy_(slot["h_oo"][: n + 1], non_blocking=True)
            codag.codag_decompress_batch_ws(slot["fm"], self.arena, slot["co"], n, self.arena,
                                            slot["oo"], slot["status"], slot["scratch"],
                                            self.scratch_bytes, stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        slot["busy"], slot["event"], slot["n"], slot["index"] = batch, ev, n, index

    def poll(self):
        """Completed batches: list of (requests, their per-chunk statuses)."""
        done = []
        for s in self.slots:
            if s["busy"] is not None and s["event"].query():
                st = s["status"][: s["n"]].cpu().numpy()
                per = [st[i:i + r.n] for r, i in zip(s["busy"], s["index"])]
                done.append((s["busy"], per))
                s["busy"] = None
        return done

    def read_output(self, r: Request) -> np.ndarray:
        return self.arena[r.out_at:r.out_at + r.out_bytes].cpu().numpy()


class Server:
    """The serving loop: arrivals -> admission -> batches -> completion."""

    def __init__(self, budget: int = 32 << 30, streams: int = 4, max_batch_chunks: int = 32768,
                 executor=None, clock=time.perf_counter, keep_results: bool = False):
        self.sched = Scheduler(budget, max_batch_chunks)
        self.ex = executor if executor is not None else GpuExecutor(budget, streams, max_batch_chunks)
        self.clock = clock
        self.keep_results = keep_results
        self.stats = Stats()

    def run(self, requests: list[Request], pinned_inputs: dict, time_limit: float = 60.0):
        """Serve `requests` (their .arrival = seconds from start, sorted);
        returns Stats.  A request's latency is its completion time, as the
        loop sees it, minus its arrival time.  The loop polls with a deadline:
        at time_limit it stops waiting, marks every request not completed by
        then timed_out, and returns Stats with status CODAG_ETIMEOUT (work
        still in flight is left to drain())."""
        t0 = self.clock()
        nxt = 0
        pending = len(requests)
        while pending and self.clock() - t0 < time_limit:
            now = self.clock() - t0
            while nxt < len(requests) and requests[nxt].arrival <= now:
                if not self.sched.arrive(requests[nxt]):
                    self.stats.rejected += 1
                    pending -= 1
                nxt += 1
            for batch, per in self.ex.poll():
                t = self.clock() - t0
                for r, st in zip(batch, per):
                    r.t_done, r.status = t, st
                    if self.keep_results:
                        r.result = self.ex.read_output(r)
                    self.sched.release(r)
                    self.stats.latencies.append(t - r.arrival)
                    self.stats.bytes_done += r.out_bytes
                    self.stats.completed += 1
                    pending -= 1
            self.sched.admit()
            if self.sched.admitted:
                slot = self.ex.free_slot()
                if slot is not None:
                    batch = self.sched.next_batch()
                    if batch:
                        for r in batch:
                            r.t_launch = self.clock() - t0
                        self.ex.launch(slot, batch, pinned_inputs)
                        self.stats.batches += 1
        self.stats.wall = self.clock() - t0
        if pending:
            for r in requests:
                if r.t_done < 0 and not r.rejected:
                    r.timed_out = True
                    self.stats.timed_out += 1
            self.stats.status = CODAG_ETIMEOUT
        return self.stats

    def drain(self):
        """Finish whatever is still in flight and forget queued requests
        (used between measurement runs)."""
        if hasattr(self.ex, "torch"):
            self.ex.torch.cuda.synchronize()
        while any(s["busy"] is not None for s in self.ex.slots):
            for batch, _ in self.ex.poll():
                for r in batch:
                    self.sched.release(r)
        for r in self.sched.admitted:
            self.sched.release(r)
        self.sched.admitted.clear()
        self.sched.waiting.clear()
        self.stats = Stats()
