"""Splitting a chunked workload across GPUs.

Chunks are independent (CODAG Sec. II-B), so several GPUs decode disjoint
chunk ranges with no exchange at all.  ``partition`` cuts the chunk list
into contiguous ranges of about equal work, measured as compressed plus
decoded bytes (the bytes a decoder reads and writes), using a prefix sum of
the offsets.  Each rank then decodes its range into its own memory; the
offsets of a range are rebased to start at 0.
"""
from __future__ import annotations

import numpy as np


def partition(comp_off: np.ndarray, out_off: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Contiguous chunk ranges [first, last) for `world` ranks, balanced by
    compressed + decoded bytes.  Ranges cover every chunk exactly once; a
    rank may get an empty range when there are fewer chunks than ranks."""
    n = len(comp_off) - 1
    work = (comp_off.astype(np.float64) + out_off.astype(np.float64))  # prefix of C + U
    total = work[-1] - work[0]
    bounds = [0]
    for r in range(1, world):
        target = work[0] + total * r / world
        b = int(np.searchsorted(work, target, side="left"))
        bounds.append(min(max(b, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def take(comp: np.ndarray, comp_off: np.ndarray, out_off: np.ndarray, first: int, last: int):
    """The chunk range [first, last) as its own workload: (comp, comp_off,
    out_off) with offsets rebased to 0."""
    ca, cb = int(comp_off[first]), int(comp_off[last])
    return (comp[ca:cb], comp_off[first:last + 1] - comp_off[first],
            out_off[first:last + 1] - out_off[first])
