"""Multi-GPU sharding logic on the CPU: balanced contiguous ranges, and a
two-rank gloo run in which every rank decodes its own range with the oracle
and the ranks' outputs together equal the whole workload (no collective on
the data path; only the final check gathers)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2307_03760_gb300.shard import partition, take


def test_partition_covers_and_balances():
    w = synth.batched(seed=2, n_chunks=500, lo=512, hi=1 << 16)
    for world in (1, 2, 3, 4, 8):
        rng = partition(w.comp_off, w.out_off, world)
        assert rng[0][0] == 0 and rng[-1][1] == w.n
        assert all(a[1] == b[0] for a, b in zip(rng, rng[1:]))
        work = [int(w.comp_off[b] - w.comp_off[a] + w.out_off[b] - w.out_off[a]) for a, b in rng]
        biggest = int(max(np.diff(w.comp_off) + np.diff(w.out_off)))
        assert max(work) - min(work) <= 2 * biggest


def test_partition_fewer_chunks_than_ranks():
    off = np.array([0, 10, 20], np.uint64)
    rng = partition(off, off, 4)
    assert sum(b - a for a, b in rng) == 2 and rng[-1][1] == 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.build_chunks([1, 2, 3, 2, 1, 3, 3, 2], [8192, 16384, 5000 // 8 * 8, 800, 64, 4096, 8, 2048],
                           seed=9)
    a, b = partition(w.comp_off, w.out_off, world)[rank]
    comp, coff, ooff = take(w.comp, w.comp_off, w.out_off, a, b)
    out, st = oracle.decode(0, comp, coff, ooff, formats=w.formats[a:b])
    assert (st == 0).all()
    parts = [None] * world
    dist.all_gather_object(parts, (a, b, out.tobytes()))
    if rank == 0:
        full, fst = oracle.decode(0, w.comp, w.comp_off, w.out_off, formats=w.formats)
        joined = b"".join(p[2] for p in sorted(parts))
        q.put(joined == full.tobytes() and sorted(p[:2] for p in parts)[0][0] == 0)
    dist.destroy_process_group()


def test_two_rank_gloo_sharded_decode():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5)
