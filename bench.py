#!/usr/bin/env python3
"""Benchmark: chunk-parallel decompression throughput on GB300.

One step = one decode of the whole workload (every chunk) through the
library's C ABI.  The headline workload is the ORC RLE v2 column (256 MiB of
signed int64 in 128 KiB chunks, 2048 chunks); ``per_format`` adds the RLE v1
column (8 MiB, 64 KiB chunks), the raw Deflate column (1 GiB, 64 KiB chunks,
zlib level 6) and the mixed batch (20,000 chunks, persistent graph-replayed
launch vs one plain launch per format), each timed the same way.

Metric: uncompressed GB/s (1e9 bytes of decoded output per second), device
time from CUDA events on the launching stream with inputs already resident
in HBM.  Inputs plus outputs exceed the 129 MB L2 in every timed workload, so
no L2 flush is inserted between steps.  ``e2e`` repeats the headline through
host buffers: pinned host -> device copy of the compressed column and its
offsets, the decode, device -> host copy of the decoded column, all inside
the timed region.  ``roofline`` relates the decode kernel's algorithmic bytes
(compressed read + decoded write + offsets) per launch to the measured HBM
copy bandwidth.  ``cpu_baseline`` times the oracle (plain single-threaded C
decoder per chunk, chunk ranges split over all host cores) on a bounded sample.

Multi-GPU (torchrun): every rank decodes its own column (weak scaling, no
collective on the data path); with ``--split`` the ranks instead decode
contiguous chunk ranges of one column, balanced by compressed + decoded
bytes (``shard.partition``; strong scaling).  The step time is the max over
ranks.
``--impl reference`` times the oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
METRIC = "uncompressed GB/s per format on 1 GB300 and % of HBM roofline; p50/p99 request latency"


def hbm_peak():
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_digest() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2307_03760_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel: str, units_per_launch: int):
    """DRAM bytes per launch from the committed ncu summary for `kernel`, if
    it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
    except Exception:
        return None
    if not rec or rec.get("source_digest") != source_digest():
        return None
    per_unit = rec["dram_bytes"] / rec["units"]
    return per_unit * units_per_launch


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dev:
    """A chunked workload resident on the device."""

    def __init__(self, w, torch, dev):
        self.w = w
        self.comp = torch.zeros(max(w.comp_bytes, 16), dtype=torch.uint8, device=dev)
        self.comp[: w.comp_bytes] = torch.from_numpy(w.comp).to(dev)
        self.coff = torch.from_numpy(w.comp_off.view(np.int64)).to(dev)
        self.ooff = torch.from_numpy(w.out_off.view(np.int64)).to(dev)
        self.fmts = torch.from_numpy(w.formats).to(dev)
        self.out = torch.empty(max(w.out_bytes, 16), dtype=torch.uint8, device=dev)
        self.status = torch.zeros(max(w.n, 1), dtype=torch.int32, device=dev)

    def alg_bytes(self) -> int:
        return self.w.comp_bytes + self.w.out_bytes + 16 * (self.w.n + 1)


def time_steps(torch, stream, fn, steps: int, warmup: int):
    """Warm up, then time `steps` calls with CUDA events on `stream`;
    returns per-step milliseconds."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def step_stats(ms):
    """mean / median / p99 of per-step milliseconds."""
    a = np.asarray(ms, dtype=np.float64)
    return {"mean": round(float(a.mean()), 5), "p50": round(float(np.percentile(a, 50)), 5),
            "p99": round(float(np.percentile(a, 99)), 5), "reps": int(a.size)}


def _cudart():
    import ctypes
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def launch_overhead(torch, stream, reps: int = 500):
    """Device time of one launch of an empty CUDA graph (the launch cost
    alone), microseconds, median over `reps` replays timed with events."""
    import ctypes
    rt = _cudart()
    if rt is None:
        return None
    g, e = ctypes.c_void_p(), ctypes.c_void_p()
    if rt.cudaGraphCreate(ctypes.byref(g), ctypes.c_uint(0)) != 0:
        return None
    if rt.cudaGraphInstantiate(ctypes.byref(e), g, ctypes.c_ulonglong(0)) != 0:
        rt.cudaGraphDestroy(g)
        return None
    sh = ctypes.c_void_p(stream.cuda_stream)
    fn = lambda: rt.cudaGraphLaunch(e, sh)  # noqa: E731
    ms = time_steps(torch, stream, fn, reps, 10)
    rt.cudaGraphExecDestroy(e)
    rt.cudaGraphDestroy(g)
    return round(1000.0 * float(np.median(ms)), 3)


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = dict(line.split(":", 1) for line in out.splitlines() if ":" in line)
        for key in ("Model name", "Vendor ID"):
            if key in fields:
                return " ".join(fields[key].split())
    except Exception:
        pass
    return os.uname().machine


def oracle_rate(w, fmt: int, seconds: float = 10.0, threads: int | None = None):
    """Oracle throughput (decoded GB/s) on a bounded sample: whole-column
    decodes split over `threads` host cores, repeated until `seconds`."""
    import oracle
    threads = threads or (os.cpu_count() or 1)
    oracle.build()
    done, t0 = 0, time.perf_counter()
    reps = 0
    while True:
        oracle.decode(fmt, w.comp, w.comp_off, w.out_off, formats=w.formats if fmt == 0 else None,
                      threads=threads)
        reps += 1
        done += w.out_bytes
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 50:
            break
    return done / el / 1e9, threads, reps, el


SCALE = 1.0  # workload size factor (profiling captures use smaller cases)


def workload(name: str, seed: int):
    if name == "rle_v1":
        return synth.rle_v1_column(seed, total=int(8 * synth.MiB * SCALE) // 65536 * 65536 or 65536)
    if name == "rle_v2":
        return synth.rle_v2_column(seed, total=int(256 * synth.MiB * SCALE) // 131072 * 131072 or 131072)
    if name == "deflate":
        return synth.deflate_column(seed, total=int(synth.GiB * SCALE) // 65536 * 65536 or 65536)
    if name == "batched":
        return synth.batched(seed, n_chunks=max(1, int(20000 * SCALE)))
    if name == "byte_rle":
        return synth.byte_rle_column(seed, total=int(64 * synth.MiB * SCALE) // 65536 * 65536 or 65536)
    if name == "bool_rle":
        return synth.bool_rle_column(seed, total=int(64 * synth.MiB * SCALE) // 65536 * 65536 or 65536)
    if name == "orc_zlib":
        return synth.orc_zlib_column(seed, total=int(synth.GiB * SCALE) // 262144 * 262144 or 262144)
    raise ValueError(name)


WORKLOAD_DESC = {
    "rle_v2": "orc_rle_v2_int64_256MiB_128KiB_chunks",
    "rle_v1": "orc_rle_v1_int64_8MiB_64KiB_chunks",
    "deflate": "raw_deflate_zlib6_1GiB_64KiB_chunks",
    "batched": "mixed_batch_20000_chunks_4KiB_1MiB",
    "byte_rle": "orc_byte_rle_64MiB_64KiB_chunks",
    "bool_rle": "orc_bool_rle_64Mi_booleans_64Ki_per_chunk",
    "orc_zlib": "orc_zlib_streams_1GiB_256KiB_streams_64KiB_blocks",
}
FMT_OF = {"rle_v1": 1, "rle_v2": 2, "deflate": 3, "byte_rle": 6, "bool_rle": 7, "orc_zlib": 8}


def run_reference(args, world, rank):
    """Oracle on the host cores, same workload / metric (rank 0 only)."""
    if rank != 0:
        return
    name = args.workload
    w = workload(name, 1)
    fmt = FMT_OF.get(name, 0)
    times = []
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    # each step: a bounded sample of whole chunks (about 2 s of host work)
    n_sample = max(1, w.n // 8) if name != "rle_v1" else w.n
    sub = slice_chunks(w, 0, n_sample)
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.decode(fmt, sub.comp, sub.comp_off, sub.out_off,
                      formats=sub.formats if fmt == 0 else None, threads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    el = sum(times)
    value = sub.out_bytes * len(times) / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * el / len(times), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64" if fmt in (1, 2) else "u8",
        "data": "synthetic", "config": {"workload": WORKLOAD_DESC[name]},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": threads,
                         "kind": "oracle",
                         "sample": f"{sub.n} of {w.n} chunks ({sub.out_bytes} decoded bytes) per step"},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def slice_chunks(w, a: int, b: int):
    ca, cb = int(w.comp_off[a]), int(w.comp_off[b])
    oa, ob = int(w.out_off[a]), int(w.out_off[b])
    return synth.Chunked(w.comp[ca:cb].copy(), (w.comp_off[a:b + 1] - w.comp_off[a]).copy(),
                         (w.out_off[a:b + 1] - w.out_off[a]).copy(), w.formats[a:b].copy(), None,
                         w.name)


def split_by_format(w):
    parts = {}
    for f in np.unique(w.formats):
        idx = np.nonzero(w.formats == f)[0]
        comp = np.concatenate([w.comp[int(w.comp_off[c]):int(w.comp_off[c + 1])] for c in idx])
        coff = np.zeros(len(idx) + 1, np.uint64)
        coff[1:] = np.cumsum(w.comp_off[idx + 1] - w.comp_off[idx])
        ooff = np.zeros(len(idx) + 1, np.uint64)
        ooff[1:] = np.cumsum(w.out_off[idx + 1] - w.out_off[idx])
        parts[int(f)] = synth.Chunked(comp, coff, ooff, w.formats[idx].copy(), None, w.name)
    return parts


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="codag", choices=["codag", "reference"])
    ap.add_argument("--workload", default="rle_v2", choices=list(WORKLOAD_DESC))
    ap.add_argument("--no-per-format", action="store_true", help="headline workload only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving sweep")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="arrival window per request rate in the serving sweep (at most 20,000 requests)")
    ap.add_argument("--serve-payloads", type=int, default=128,
                    help="distinct request payloads the serving sweep draws from")
    ap.add_argument("--parts", type=int, default=0,
                    help="parts per RLE chunk (0 = library default)")
    ap.add_argument("--no-tuning", action="store_true",
                    help="ignore the committed autotuner table")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="workload size factor; 1.0 is the measured configuration")
    ap.add_argument("--split", action="store_true",
                    help="ranks decode balanced ranges of one column (strong scaling) "
                         "instead of a column each")
    args = ap.parse_args()
    global SCALE
    SCALE = args.scale
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, world, rank)
        return

    import torch
    import paper_2307_03760_gb300 as codag

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    codag.lib()
    from paper_2307_03760_gb300 import autotune
    tuned = autotune.apply(n_chunks=None, family=args.workload) if not args.no_tuning else {}
    if args.parts:
        codag.codag_set_parts_per_chunk(args.parts)
    stream = torch.cuda.current_stream()
    peak, peak_kind = hbm_peak()

    name = args.workload
    if args.split:
        from paper_2307_03760_gb300 import shard
        whole = workload(name, 1)
        first, last = shard.partition(whole.comp_off, whole.out_off, world)[rank]
        w = slice_chunks(whole, first, last)
        job_bytes = whole.out_bytes
    else:
        w = workload(name, 1 + rank)
        job_bytes = world * w.out_bytes
    d = Dev(w, torch, dev)

    # arguments resolved once (raw pointers and stream handle), so that a step
    # costs the host one library call
    sh = stream.cuda_stream
    pb = (d.fmts.data_ptr(), d.comp.data_ptr(), d.coff.data_ptr(), w.n, d.out.data_ptr(),
          d.ooff.data_ptr(), d.status.data_ptr())

    def step():
        if name == "batched":
            codag.codag_decompress_batch(*pb, stream=sh)
        else:
            codag.codag_decompress(FMT_OF[name], *pb[1:6], stream=sh)

    # correctness of the timed configuration: every chunk decodes OK
    step()
    torch.cuda.synchronize()
    st = d.status.cpu().numpy()[: w.n] if name == "batched" else codag.codag_last_chunk_status(w.n)
    if (np.asarray(st) != 0).any():
        raise SystemExit(f"decode reported chunk errors: {np.unique(st)}")

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = codag.codag_kernel_launches()
    with ClockSampler(local) as clk:
        ms = time_steps(torch, stream, step, args.steps, args.warmup)
    launches = codag.codag_kernel_launches() - launches0
    gpu_launches = launches * args.steps // (args.steps + args.warmup)
    total_ms = sum(ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    value = job_bytes * args.steps / (total_ms / 1e3) / 1e9
    # one decode launch per step for the RLE columns; the Deflate column's
    # step is its two passes (Huffman, then LZ77) and the batch step the
    # persistent kernel with its ordering and status kernels, timed together
    kernel_ms = statistics.mean(ms)
    achieved = d.alg_bytes() / (kernel_ms / 1e3) / 1e9
    kernel = {"rle_v1": "rle_v1_kernel", "rle_v2": "rle_v2_kernel", "deflate": "inflate_huffman_kernel",
              "batched": "batch_kernel", "byte_rle": "byte_rle_cta_kernel",
              "bool_rle": "byte_rle_cta_kernel", "orc_zlib": "orc_zlib_kernel"}[name]
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                "nominal_peak": NOMINAL_HBM_GBS,
                "traffic": traffic_from_profile(kernel, w.n), "kernel": kernel,
                "timed": "the whole step" if name in ("deflate", "batched") else "the kernel (one launch per step)",
                "algorithmic_bytes_per_launch": d.alg_bytes()}

    # end to end through host buffers (pinned), copies inside the timed region
    h_comp = torch.from_numpy(w.comp).pin_memory() if w.comp_bytes else torch.zeros(16, dtype=torch.uint8).pin_memory()
    h_coff = torch.from_numpy(w.comp_off.view(np.int64)).pin_memory()
    h_ooff = torch.from_numpy(w.out_off.view(np.int64)).pin_memory()
    h_out = torch.empty(max(w.out_bytes, 16), dtype=torch.uint8).pin_memory()

    h_status = torch.empty(max(w.n, 1), dtype=torch.int32).pin_memory()

    def e2e_step():
        if name == "batched":  # the batch call takes device buffers: copies around it
            d.comp[: w.comp_bytes].copy_(h_comp[: w.comp_bytes], non_blocking=True)
            d.coff.copy_(h_coff, non_blocking=True)
            d.ooff.copy_(h_ooff, non_blocking=True)
            step()
            h_out[: w.out_bytes].copy_(d.out[: w.out_bytes], non_blocking=True)
            h_status[: w.n].copy_(d.status[: w.n], non_blocking=True)
        else:  # host-to-host call: slice copies overlap the decode
            codag.codag_decompress_host(FMT_OF[name], h_comp, h_coff, w.n, h_out, h_ooff,
                                        d.comp, d.out, h_status)

    e2e_ms = time_steps(torch, stream, e2e_step, max(3, args.steps // 2), 2)
    e2e_t = sum(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e_t], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_t = float(t.item())
    e2e_val = job_bytes * len(e2e_ms) / (e2e_t / 1e3) / 1e9
    torch.cuda.synchronize()
    ok = np.array_equal(h_out[: w.out_bytes].numpy(), d.out[: w.out_bytes].cpu().numpy()) and \
        bool((h_status[: w.n].numpy() == 0).all())

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "strong" if args.split else "weak", "vs_baseline": None,
        "dtype": "int64" if name in ("rle_v1", "rle_v2") else "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[name] + ("" if SCALE == 1.0 else f"_scaled_{SCALE}"), "chunks": w.n, "compressed_bytes": w.comp_bytes,
                   "uncompressed_bytes": w.out_bytes, "ratio": round(w.comp_bytes / w.out_bytes, 4),
                   "l2": "inputs+outputs larger than L2 (no flush)", "seed": 1,
                   "parallelism": (f"chunk-parallel x{world} (one column split into balanced chunk ranges)"
                                   if args.split else f"chunk-parallel x{world} (independent columns per GPU)"),
                   "parts_per_chunk": codag.codag_get_parts_per_chunk() or "auto",
                   **({"batch_ctas_per_sm": codag.codag_get_batch_ctas_per_sm() or "all that fit",
                       "staging_depth": "%d x %d bytes per warp" % codag.codag_get_batch_staging(),
                       "chunk_mapping": "RLE chunk of 2^b bytes on min(2^(b-%d), %d) warps"
                                        % codag.codag_get_batch_split()}
                      if name == "batched" else {}),
                   "tuning": tuned},
        "e2e": {"value": round(e2e_val, 2), "unit": "GB/s",
                "h2d_bytes_per_step": w.comp_bytes + 16 * (w.n + 1),
                "d2h_bytes_per_step": w.out_bytes + 4 * w.n, "output_checked": bool(ok),
                "api": "codag_decompress_batch between copies" if name == "batched"
                       else "codag_decompress_host (16 MiB slices, copies overlapped)"},
        "roofline": roofline,
        "step_ms": step_stats(ms),
        "launch_overhead_us": launch_overhead(torch, stream) if rank == 0 else None,
        "gpu_launches": int(gpu_launches),
        "clocks": clk.summary(),
    }

    if rank == 0 and world == 1 and not args.no_per_format:
        line["per_format"] = per_format(torch, codag, dev, stream, peak, name, w, d, value, achieved)

    if rank == 0 and world == 1 and not args.no_serving:
        line["serving"] = serving(torch, args.serve_seconds, args.serve_payloads)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, reps, el = oracle_rate(w, FMT_OF.get(name, 0), seconds=10.0)
        # one core, on a slice of the column (about 3 s)
        sub1 = slice_chunks(w, 0, max(1, w.n // 16))
        rate1, _, reps1, el1 = oracle_rate(sub1, FMT_OF.get(name, 0), seconds=3.0, threads=1)
        line["cpu_baseline"] = {"value": round(rate, 3), "unit": "GB/s", "cores": threads,
                                "kind": "oracle", "cpu": cpu_model(),
                                "sample": f"{reps} whole-column decode(s) of the same workload "
                                          f"({w.out_bytes} bytes each) in {el:.1f} s",
                                "single_thread": {"value": round(rate1, 3), "unit": "GB/s", "cores": 1,
                                                  "sample": f"{reps1} decode(s) of the first {sub1.n} "
                                                            f"chunks ({sub1.out_bytes} bytes) in {el1:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def serving(torch, seconds: float, n_payloads: int = 128):
    """Continuous-batching server under Poisson arrivals: requests of 1-256
    chunks of one random format, 64 KiB-64 MiB decoded, 32 GiB HBM budget.
    Latency = arrival -> completion seen by the host, including the copy of
    the request's compressed bytes from pinned host memory."""
    from paper_2307_03760_gb300.serve import Request, Server
    pool = synth.serving_pool(seed=1, n_payloads=n_payloads)
    pinned = [torch.from_numpy(w.comp).pin_memory() for w in pool]
    mean_bytes = float(np.mean([w.out_bytes for w in pool]))
    srv = Server(budget=32 << 30, streams=4, max_batch_chunks=32768)
    # warm the path once
    warm = [Request(0, pool[0].formats, pool[0].comp, pool[0].comp_off, pool[0].out_off, 0.0)]
    srv.run(warm, {0: pinned[0]}, time_limit=10.0)
    srv.drain()
    out = {"payloads": len(pool), "mean_request_bytes": int(mean_bytes),
           "budget_bytes": 32 << 30, "streams": 4, "rates": {}}
    for lam in (1000, 2000, 5000, 10000, 20000, 50000):
        times, pick = synth.poisson_arrivals(1, float(lam), seconds, len(pool))
        times, pick = times[:20000], pick[:20000]
        reqs = [Request(i, pool[p].formats, pool[p].comp, pool[p].comp_off, pool[p].out_off,
                        float(t)) for i, (t, p) in enumerate(zip(times, pick))]
        inputs = {r.rid: pinned[p] for r, p in zip(reqs, pick)}
        window = float(times[-1]) if len(times) else seconds  # arrivals end here
        # after the last arrival the loop drains: allow the offered bytes at 25 GB/s
        offered = float(sum(pool[p].out_bytes for p in pick))
        st = srv.run(reqs, inputs, time_limit=window + 4.0 + offered / 25e9)
        summ = st.summary()
        summ["offered_GBps"] = round(lam * mean_bytes / 1e9, 2)
        summ["requests"] = len(reqs)
        summ["arrival_window_s"] = round(window, 3)
        summ["errors"] = int(sum(int((r.status != 0).any()) for r in reqs if r.status is not None))
        out["rates"][str(lam)] = summ
        srv.drain()
    return out


def per_format(torch, codag, dev, stream, peak, headline, hw, hd, hvalue, hach):
    res = {headline: {"GBps": round(hvalue, 2), "hbm_frac": round(hach / peak, 4),
                      "hbm_frac_of_nominal": round(hach / NOMINAL_HBM_GBS, 4)}}
    for name in ("rle_v1", "deflate", "byte_rle", "bool_rle", "orc_zlib"):
        if name == headline:
            continue
        w = workload(name, 1)
        d = Dev(w, torch, dev)
        fmt = FMT_OF[name]
        # this family's tuned warps per chunk (auto if none)
        from paper_2307_03760_gb300 import autotune
        codag.codag_set_parts_per_chunk(0)
        autotune.apply(n_chunks=w.n, family="byte_rle" if name == "bool_rle" else name)
        args = (fmt, d.comp.data_ptr(), d.coff.data_ptr(), w.n, d.out.data_ptr(), d.ooff.data_ptr())
        sh = stream.cuda_stream
        fn = lambda: codag.codag_decompress(*args, stream=sh)  # noqa: E731
        fn()
        torch.cuda.synchronize()
        st = codag.codag_last_chunk_status(w.n)
        reps = 10 if name in ("deflate", "orc_zlib") else 400 if name == "rle_v1" else 100
        ms = time_steps(torch, stream, fn, reps, 3)
        t = statistics.median(ms)
        res[name] = {"GBps": round(w.out_bytes / (t / 1e3) / 1e9, 2),
                     "hbm_frac": round(d.alg_bytes() / (t / 1e3) / 1e9 / peak, 4),
                     "hbm_frac_of_nominal": round(d.alg_bytes() / (t / 1e3) / 1e9 / NOMINAL_HBM_GBS, 4),
                     "ms": round(t, 4), "step_ms": step_stats(ms),
                     "chunks": w.n, "ratio": round(w.comp_bytes / w.out_bytes, 4),
                     "all_ok": bool((st == 0).all()), "workload": WORKLOAD_DESC[name]}
        del d
    codag.codag_set_parts_per_chunk(0)
    # mixed batch: persistent graph-captured launch vs one plain launch per format
    w = workload("batched", 1)
    d = Dev(w, torch, dev)
    g = codag.BatchGraph(d.fmts, d.comp, d.coff, w.n, d.out, d.ooff, d.status)
    ms_g = time_steps(torch, stream, g.launch, 10, 3)
    ok_g = bool((d.status.cpu().numpy()[: w.n] == 0).all())
    parts = split_by_format(w)
    devs = {f: Dev(p, torch, dev) for f, p in parts.items()}

    # each plain launch with its family's tuned warps per chunk
    from paper_2307_03760_gb300 import autotune
    tuned_parts = {}
    if os.path.exists(autotune.DEFAULT_TABLE):
        with open(autotune.DEFAULT_TABLE) as fh:
            rp = json.load(fh).get("rle_parts", {})
        tuned_parts = {1: rp.get("rle_v1", {}).get("best", 0), 2: rp.get("rle_v2", {}).get("best", 0)}

    def three():
        for f, pd in devs.items():
            codag.codag_set_parts_per_chunk(int(tuned_parts.get(f, 0)))
            codag.codag_decompress(f, pd.comp, pd.coff, pd.w.n, pd.out, pd.ooff)
        codag.codag_set_parts_per_chunk(0)

    ms_p = time_steps(torch, stream, three, 10, 3)
    tg, tp = statistics.median(ms_g), statistics.median(ms_p)
    res["batched"] = {"graph_persistent_GBps": round(w.out_bytes / (tg / 1e3) / 1e9, 2),
                      "per_format_launches_GBps": round(w.out_bytes / (tp / 1e3) / 1e9, 2),
                      "speedup": round(tp / tg, 3), "ms_graph": round(tg, 3), "ms_plain": round(tp, 3),
                      "hbm_frac": round(d.alg_bytes() / (tg / 1e3) / 1e9 / peak, 4),
                      "chunks": w.n, "uncompressed_bytes": w.out_bytes, "all_ok": ok_g,
                      "workload": WORKLOAD_DESC["batched"]}
    g.destroy()
    return res


if __name__ == "__main__":
    main()
