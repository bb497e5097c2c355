"""The bench's reference arm (the FP64 oracle timed on the host cores) runs
without a GPU: one JSON line with the contract's keys, on the same metric,
unit and workload (512 x 512, sigma 4 px, alpha 1e-2) as the CUDA arm, and a
cpu_baseline / e2e describing the run itself.  The CUDA arm's keys are checked on the GPU by running it."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    wl = bench.WORKLOADS["c3"]
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "RHS/s"
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"] == wl["name"]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == d["unit"] and cb["sample"]
    # the sample is one oracle cycle per step, scaled by the oracle's own
    # cycle count to 1e-6, stored for this workload
    assert wl["name"] in json.load(open(os.path.join(ROOT, "tests", "golden",
                                                      "oracle_cycles.json")))
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
