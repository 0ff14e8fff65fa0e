"""Autotuner for the launch shapes the library leaves open.

Three knobs: parts per RLE chunk for the plain RLE calls (warps cooperating
on one chunk; ``codag_set_parts_per_chunk``), resident CTAs per SM of the
persistent batch kernel (decoders per SM; ``codag_set_batch_ctas_per_sm``),
and the input staging of the one-warp-per-chunk decoders (shared-memory TMA
ring or register ring; ``codag_set_input_staging``) for Deflate and byte RLE.
``sweep`` times every candidate on a workload with CUDA events and keeps the
fastest; ``tune`` runs the sweeps and writes a table, ``apply`` loads a
table into the library.  The selection is separated from the timing so it
can be checked without a GPU.
"""
from __future__ import annotations

import json
import os
import statistics

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuning_gb300.json")


def choose(timings: dict) -> tuple:
    """Fastest candidate by median time; ties go to the smaller value
    (fewer warps per chunk / fewer CTAs per SM leave more room to others)."""
    best = None
    for cand, times in sorted(timings.items()):
        m = statistics.median(times)
        if best is None or m < best[1] * (1 - 1e-9):
            best = (cand, m)
    return best


def sweep(run, candidates, setter, reps: int = 7, warmup: int = 2, timer=None) -> dict:
    """Time `run()` for every candidate (set through `setter`); returns
    {candidate: [ms, ...]}."""
    out = {}
    for c in candidates:
        setter(c)
        for _ in range(warmup):
            run()
        out[c] = [timer(run) for _ in range(reps)]
    return out


def _event_timer(torch):
    def t(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    return t


def tune(path: str = DEFAULT_TABLE, seed: int = 1) -> dict:
    import numpy as np
    import torch

    import synth
    import paper_2307_03760_gb300 as codag
    dev = torch.device("cuda", 0)
    timer = _event_timer(torch)

    def upload(w):
        comp = torch.zeros(max(w.comp_bytes, 16), dtype=torch.uint8, device=dev)
        comp[: w.comp_bytes] = torch.from_numpy(w.comp).to(dev)
        return (comp, torch.from_numpy(w.comp_off.view(np.int64)).to(dev),
                torch.from_numpy(w.out_off.view(np.int64)).to(dev),
                torch.from_numpy(w.formats).to(dev),
                torch.empty(max(w.out_bytes, 16), dtype=torch.uint8, device=dev),
                torch.zeros(max(w.n, 1), dtype=torch.int32, device=dev))

    table = {"device": torch.cuda.get_device_name(0), "rle_parts": {}, "sweeps": {}}
    for name, w in (("rle_v1", synth.rle_v1_column(seed)), ("rle_v2", synth.rle_v2_column(seed)),
                    ("byte_rle", synth.byte_rle_column(seed))):
        comp, coff, ooff, _, out, _ = upload(w)
        fmt = int(w.formats[0])
        run = lambda: codag.codag_decompress(fmt, comp, coff, w.n, out, ooff)  # noqa: E731
        t = sweep(run, list(range(1, 17)), codag.codag_set_parts_per_chunk, timer=timer)
        best, ms = choose(t)
        table["rle_parts"][name] = {"chunks": w.n, "best": best, "ms": round(ms, 4)}
        table["sweeps"][f"{name}_parts"] = {str(k): round(statistics.median(v), 4) for k, v in t.items()}
    codag.codag_set_parts_per_chunk(0)
    # input staging of the one-warp-per-chunk decoders (0: shared ring, 1: registers)
    table["input_staging"] = {}
    for name, w in (("deflate", synth.deflate_column(seed, total=256 * synth.MiB)),
                    ("byte_rle", synth.byte_rle_column(seed))):
        comp, coff, ooff, _, out, _ = upload(w)
        fmt = int(w.formats[0])
        run = lambda: codag.codag_decompress(fmt, comp, coff, w.n, out, ooff)  # noqa: E731
        t = sweep(run, [0, 1], lambda m: codag.codag_set_input_staging(fmt, m), reps=5, timer=timer)
        best, ms = choose(t)
        table["input_staging"][name] = {"format": fmt, "best": best, "ms": round(ms, 4)}
        table["sweeps"][f"{name}_input_staging"] = {str(k): round(statistics.median(v), 4) for k, v in t.items()}
        codag.codag_set_input_staging(fmt, 0)
    # the full mixed batch: a sample of it would be dominated by its largest
    # chunk and favour too few CTAs
    w = synth.batched(seed)
    comp, coff, ooff, fm, out, st = upload(w)
    run = lambda: codag.codag_decompress_batch(fm, comp, coff, w.n, out, ooff, st)  # noqa: E731
    t = sweep(run, [1, 2, 3, 4, 5, 6, 8], codag.codag_set_batch_ctas_per_sm, reps=3, warmup=1,
              timer=timer)
    best, ms = choose(t)
    table["batch_ctas_per_sm"] = {"best": best, "ms": round(ms, 3), "chunks": w.n}
    table["sweeps"]["batch_ctas_per_sm"] = {str(k): round(statistics.median(v), 3) for k, v in t.items()}
    codag.codag_set_batch_ctas_per_sm(0)
    with open(path, "w") as f:
        json.dump(table, f, indent=1)
    return table


def apply(path: str = DEFAULT_TABLE, n_chunks: int | None = None, family: str = "rle_v2") -> dict:
    """Load a tuning table into the library: batch CTAs per SM, and parts per
    RLE chunk for `family` when the tuned chunk count matches `n_chunks`.
    Returns what was set ({} if there is no table)."""
    import paper_2307_03760_gb300 as codag
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        table = json.load(f)
    done = {}
    b = table.get("batch_ctas_per_sm", {}).get("best")
    if b:
        codag.codag_set_batch_ctas_per_sm(int(b))
        done["batch_ctas_per_sm"] = int(b)
    p = table.get("rle_parts", {}).get(family)
    if p and (n_chunks is None or p.get("chunks") == n_chunks):
        codag.codag_set_parts_per_chunk(int(p["best"]))
        done["parts_per_chunk"] = int(p["best"])
    for name, e in table.get("input_staging", {}).items():
        codag.codag_set_input_staging(int(e["format"]), int(e["best"]))
        if int(e["format"]) == 6:  # boolean RLE runs the same decoder
            codag.codag_set_input_staging(7, int(e["best"]))
        done[f"input_staging_{name}"] = int(e["best"])
    return done


if __name__ == "__main__":
    import sys
    print(json.dumps(tune(sys.argv[1] if len(sys.argv) > 1 else DEFAULT_TABLE), indent=1))
