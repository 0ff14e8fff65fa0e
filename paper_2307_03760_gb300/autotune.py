"""Autotuner for the launch shapes the library leaves open.

Knobs: parts per RLE chunk for the plain RLE calls (warps cooperating on one
chunk; ``codag_set_parts_per_chunk``); the input staging of the
one-warp-per-chunk decoders (shared-memory TMA ring or register ring;
``codag_set_input_staging``) for Deflate and byte RLE; and three of the
persistent batch kernel, tuned on the full mixed batch: its input-ring shape
(slot bytes x slots per warp, ``staging_depth``;
``codag_set_batch_staging``) jointly with its resident CTAs per SM
(``codag_set_batch_ctas_per_sm``), then the rule that splits large RLE
chunks over several warps (``chunk_mapping``; ``codag_set_batch_split``).
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


def choose(timings: dict, rel_tol: float = 0.01) -> tuple:
    """(candidate, its median time): the fastest by median, where candidates
    within rel_tol of the fastest count as ties, which go to the smallest
    candidate (fewer warps per chunk or CTAs per SM leave room to others,
    and settings that launch the same thing, such as CTA counts above what
    fits on an SM, only differ by noise)."""
    med = {c: statistics.median(t) for c, t in timings.items()}
    m0 = min(med.values())
    for c in sorted(med):
        if med[c] <= m0 * (1 + rel_tol):
            return c, med[c]


def _unkey(k: str):
    return tuple(int(v) for v in k.split("x")) if "x" in k else int(k)


def reselect(table: dict) -> dict:
    """Recompute a table's choices from its recorded sweeps (medians, ms)
    with `choose`; tune() ends with this, and it re-applies a changed
    selection rule to measurements already taken."""
    sw = table.get("sweeps", {})
    for name, e in table.get("rle_parts", {}).items():
        if f"{name}_parts" in sw:
            c, ms = choose({_unkey(k): [v] for k, v in sw[f"{name}_parts"].items()})
            e["best"], e["ms"] = c, round(ms, 4)
    for name, e in table.get("input_staging", {}).items():
        if f"{name}_input_staging" in sw:
            c, ms = choose({_unkey(k): [v] for k, v in sw[f"{name}_input_staging"].items()})
            e["best"], e["ms"] = c, round(ms, 4)
    if "batch_staging_x_ctas" in sw and "staging_depth" in table:
        (slot, slots, ctas), ms = choose({_unkey(k): [v] for k, v in sw["batch_staging_x_ctas"].items()})
        table["staging_depth"].update(best=[slot, slots], ms=round(ms, 3))
        table["batch_ctas_per_sm"].update(best=ctas, ms=round(ms, 3))
    if "batch_split" in sw and "chunk_mapping" in table:
        (lg, mx), ms = choose({_unkey(k): [v] for k, v in sw["batch_split"].items()})
        table["chunk_mapping"].update(best=[lg, mx], ms=round(ms, 3))
    return table


# RLE split rules offered to the batch sweep: (split_log2, max_parts)
SPLIT_RULES = [(s, m) for s in (13, 14, 15, 16, 17, 18) for m in (8, 16, 32)] + [(16, 1)]
BATCH_CTAS = [1, 2, 3, 4, 5, 6, 8, 9]


def sweep(run, candidates, setter, reps: int = 7, warmup: int = 2, timer=None, sync=None) -> dict:
    """Time `run()` for every candidate (set through `setter`); returns
    {candidate: [ms, ...]}.  sync (if given) runs after each warm-up call, so
    that what a call learns for the next one (the Deflate command pool size)
    is in place before the timed calls."""
    out = {}
    for c in candidates:
        setter(c)
        for _ in range(warmup):
            run()
            if sync:
                sync()
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


def _key(c) -> str:
    return "x".join(str(v) for v in c) if isinstance(c, tuple) else str(c)


def tune_batch(table: dict, seed: int = 1) -> dict:
    """The batch kernel's knobs on the full mixed batch (a sample of it would
    be dominated by its largest chunk and favour too few CTAs): ring shape x
    CTAs per SM jointly, then the RLE split rule at the best pair."""
    import numpy as np
    import torch

    import synth
    import paper_2307_03760_gb300 as codag
    dev = torch.device("cuda", 0)
    timer = _event_timer(torch)
    w = synth.batched(seed)
    comp = torch.zeros(max(w.comp_bytes, 16), dtype=torch.uint8, device=dev)
    comp[: w.comp_bytes] = torch.from_numpy(w.comp).to(dev)
    coff = torch.from_numpy(w.comp_off.view(np.int64)).to(dev)
    ooff = torch.from_numpy(w.out_off.view(np.int64)).to(dev)
    fm = torch.from_numpy(w.formats).to(dev)
    out = torch.empty(max(w.out_bytes, 16), dtype=torch.uint8, device=dev)
    st = torch.zeros(max(w.n, 1), dtype=torch.int32, device=dev)
    run = lambda: codag.codag_decompress_batch(fm, comp, coff, w.n, out, ooff, st)  # noqa: E731

    def set_pair(c):
        slot, slots, ctas = c
        codag.codag_set_batch_staging(slot, slots)
        codag.codag_set_batch_ctas_per_sm(ctas)

    pairs = [(slot, slots, k) for slot, slots in codag.codag_batch_staging_shapes() for k in BATCH_CTAS]
    try:
        codag.codag_set_batch_split(0, 0)
        t = sweep(run, pairs, set_pair, reps=3, warmup=1, timer=timer)
        (slot, slots, ctas), ms = choose(t)
        table["staging_depth"] = {"best": [slot, slots], "ms": round(ms, 3), "chunks": w.n}
        table["batch_ctas_per_sm"] = {"best": ctas, "ms": round(ms, 3), "chunks": w.n}
        table["sweeps"]["batch_staging_x_ctas"] = {_key(k): round(statistics.median(v), 3)
                                                   for k, v in t.items()}
        set_pair((slot, slots, ctas))
        t = sweep(run, SPLIT_RULES, lambda c: codag.codag_set_batch_split(*c), reps=3, warmup=1,
                  timer=timer)
        (lg, mx), ms = choose(t)
        table["chunk_mapping"] = {"best": [lg, mx], "ms": round(ms, 3), "chunks": w.n,
                                  "rule": "an RLE chunk of 2^b bytes runs on min(2^(b - split_log2), "
                                          "max_parts) warps when b > split_log2"}
        table["sweeps"]["batch_split"] = {_key(k): round(statistics.median(v), 3) for k, v in t.items()}
    finally:
        codag.codag_set_batch_staging(0, 0)
        codag.codag_set_batch_ctas_per_sm(0)
        codag.codag_set_batch_split(0, 0)
    return table


def tune(path: str = DEFAULT_TABLE, seed: int = 1, only_batch: bool = False) -> dict:
    """Run the sweeps and write the table to `path`.  only_batch: keep the
    other entries of an existing table and re-tune the batch knobs alone."""
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

    if only_batch and os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
        table.setdefault("sweeps", {})
        table["device"] = torch.cuda.get_device_name(0)
        tune_batch(table, seed)
        reselect(table)
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
        return table
    table = {"device": torch.cuda.get_device_name(0), "rle_parts": {}, "sweeps": {}}
    for name, w in (("rle_v1", synth.rle_v1_column(seed)), ("rle_v2", synth.rle_v2_column(seed)),
                    ("byte_rle", synth.byte_rle_column(seed))):
        comp, coff, ooff, _, out, _ = upload(w)
        fmt = int(w.formats[0])
        run = lambda: codag.codag_decompress(fmt, comp, coff, w.n, out, ooff)  # noqa: E731
        t = sweep(run, list(range(1, 17)), codag.codag_set_parts_per_chunk, timer=timer,
                  sync=torch.cuda.synchronize)
        best, ms = choose(t)
        table["rle_parts"][name] = {"chunks": w.n, "best": best, "ms": round(ms, 4)}
        table["sweeps"][f"{name}_parts"] = {str(k): round(statistics.median(v), 4) for k, v in t.items()}
    codag.codag_set_parts_per_chunk(0)
    # input staging of Deflate (0: two passes, 1: one warp per chunk through a
    # register ring) and byte RLE (0: shared ring, 1: registers), on the full
    # columns: the Huffman pass gives each chunk one lane, so it needs tens of
    # thousands of chunks to fill the GPU, and a smaller column would favour
    # the one-warp decoder
    table["input_staging"] = {}
    for name, w in (("deflate", synth.deflate_column(seed)),
                    ("byte_rle", synth.byte_rle_column(seed))):
        comp, coff, ooff, _, out, _ = upload(w)
        fmt = int(w.formats[0])
        run = lambda: codag.codag_decompress(fmt, comp, coff, w.n, out, ooff)  # noqa: E731
        t = sweep(run, [0, 1], lambda m: codag.codag_set_input_staging(fmt, m), reps=5, timer=timer,
                  sync=torch.cuda.synchronize)
        best, ms = choose(t)
        table["input_staging"][name] = {"format": fmt, "best": best, "ms": round(ms, 4)}
        table["sweeps"][f"{name}_input_staging"] = {str(k): round(statistics.median(v), 4) for k, v in t.items()}
        codag.codag_set_input_staging(fmt, 0)
    tune_batch(table, seed)
    reselect(table)
    with open(path, "w") as f:
        json.dump(table, f, indent=1)
    return table


def apply(path: str = DEFAULT_TABLE, n_chunks: int | None = None, family: str = "rle_v2") -> dict:
    """Load a tuning table into the library: the batch kernel's CTAs per SM,
    ring shape and RLE split rule, the input staging of the one-warp
    decoders, and parts per RLE chunk for `family` when the tuned chunk count
    matches `n_chunks`.  Returns what was set ({} if there is no table)."""
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
    d = table.get("staging_depth", {}).get("best")
    if d:
        codag.codag_set_batch_staging(int(d[0]), int(d[1]))
        done["staging_depth"] = [int(d[0]), int(d[1])]
    m = table.get("chunk_mapping", {}).get("best")
    if m:
        codag.codag_set_batch_split(int(m[0]), int(m[1]))
        done["chunk_mapping"] = [int(m[0]), int(m[1])]
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
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    path = args[0] if args else DEFAULT_TABLE
    if "--reselect" in sys.argv:  # no GPU: re-apply `choose` to the recorded sweeps
        with open(path) as f:
            t = reselect(json.load(f))
        with open(path, "w") as f:
            json.dump(t, f, indent=1)
        print(json.dumps({k: v for k, v in t.items() if k != "sweeps"}, indent=1))
    else:
        print(json.dumps(tune(path, only_batch="--only-batch" in sys.argv), indent=1))
