"""Device helpers for the GPU tests: upload a chunked workload, run the
library through its C ABI, bring outputs and statuses back."""
from __future__ import annotations

import numpy as np
import torch

import paper_2307_03760_gb300 as codag

DEV = torch.device("cuda:0")


def dev_u8(a: np.ndarray, min_bytes: int = 16) -> torch.Tensor:
    t = torch.zeros(max(a.size, min_bytes), dtype=torch.uint8, device=DEV)
    if a.size:
        t[: a.size] = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return t


def dev_u64(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(DEV)


def pack(chunks: list[bytes]):
    """Concatenate byte strings into (comp, comp_off)."""
    off = np.zeros(len(chunks) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(c) for c in chunks]) if chunks else []
    comp = np.frombuffer(b"".join(chunks), dtype=np.uint8).copy() if chunks else np.zeros(0, np.uint8)
    return comp, off


def run_plain(fmt: int, comp: np.ndarray, comp_off: np.ndarray, out_off: np.ndarray,
              out_shift: int = 0):
    """codag_decompress; returns (out bytes, per-chunk status)."""
    n = len(comp_off) - 1
    total = int(out_off[-1]) if n else 0
    d_comp, d_coff, d_ooff = dev_u8(comp), dev_u64(comp_off), dev_u64(out_off)
    out = torch.full((total + out_shift + 64,), 0xA5, dtype=torch.uint8, device=DEV)
    codag.codag_decompress(fmt, d_comp, d_coff, n, out.data_ptr() + out_shift, d_ooff)
    status = codag.codag_last_chunk_status(n)
    return out[out_shift: out_shift + total].cpu().numpy(), status


def run_sizes(fmt: int, comp: np.ndarray, comp_off: np.ndarray):
    n = len(comp_off) - 1
    sizes = torch.zeros(max(n, 1), dtype=torch.int64, device=DEV)
    codag.codag_decompressed_sizes(fmt, dev_u8(comp), dev_u64(comp_off), n, sizes)
    status = codag.codag_last_chunk_status(n)
    return sizes[:n].cpu().numpy().view(np.uint64), status


def run_batch(formats: np.ndarray, comp: np.ndarray, comp_off: np.ndarray, out_off: np.ndarray,
              graph: bool = False, replays: int = 1):
    n = len(comp_off) - 1
    total = int(out_off[-1])
    d_fmt = dev_u8(np.asarray(formats, dtype=np.uint8))
    d_comp, d_coff, d_ooff = dev_u8(comp), dev_u64(comp_off), dev_u64(out_off)
    out = torch.full((total + 64,), 0xA5, dtype=torch.uint8, device=DEV)
    st = torch.full((max(n, 1),), -1, dtype=torch.int32, device=DEV)
    if graph:
        g = codag.BatchGraph(d_fmt, d_comp, d_coff, n, out, d_ooff, st)
        for _ in range(replays):
            out.fill_(0xA5)
            st.fill_(-1)
            g.launch()
        torch.cuda.synchronize()
        g.destroy()
    else:
        codag.codag_decompress_batch(d_fmt, d_comp, d_coff, n, out, d_ooff, st)
    torch.cuda.synchronize()
    return out[:total].cpu().numpy(), st[:n].cpu().numpy()


def assert_parity(fmt, comp, comp_off, out_off, got, gstatus, formats=None, threads=8):
    """GPU vs oracle: equal status per chunk; equal bytes on every OK chunk."""
    import oracle
    exp, estatus = oracle.decode(fmt, comp, comp_off, out_off, formats=formats, threads=threads)
    bad = np.nonzero(np.asarray(gstatus) != estatus)[0]
    assert bad.size == 0, f"status mismatch on {bad.size} chunks, first {bad[:8]}: " \
        f"gpu {np.asarray(gstatus)[bad[:8]]} oracle {estatus[bad[:8]]}"
    ok = estatus == 0
    if ok.all():
        if not np.array_equal(got, exp):
            diff = np.nonzero(got != exp)[0]
            c = np.searchsorted(out_off, diff[0], side="right") - 1
            raise AssertionError(f"{diff.size} bytes differ, first at {diff[0]} (chunk {c})")
    else:
        for c in np.nonzero(ok)[0]:
            a, b = int(out_off[c]), int(out_off[c + 1])
            assert np.array_equal(got[a:b], exp[a:b]), f"chunk {c} differs"
    return estatus
