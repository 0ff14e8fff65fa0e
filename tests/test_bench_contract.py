"""bench.py's reference arm on the CPU: the one JSON line it prints keeps
the contract (metric, unit, value, the oracle's core count and sample, an
end-to-end figure with no copies), at a small scale so that it runs in
seconds; and the committed ncu traffic figures are per-launch byte counts
of the kernels the bench reports."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["rle_v2", "rle_v1", "deflate"])
def test_reference_line(workload):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "3", "--scale", "0.02"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "GB/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["n_gpus"] == 1
    assert line["steps"] == 1 and line["warmup"] >= 3
    assert line["data"] == "synthetic" and line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "chunks" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_committed_traffic_entries():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    for kernel in ("rle_v2_kernel", "rle_v1_kernel", "inflate_huffman_kernel", "inflate_lz77_kernel", "batch_kernel"):
        e = t[kernel]
        assert e["dram_bytes"] == e["dram_read"] + e["dram_write"] > 0
        assert e["units"] > 0 and e["workload"] and e["command"].startswith("ncu ")
        assert "--clock-control none" in e["command"]
        assert len(e["source_digest"]) == 16
