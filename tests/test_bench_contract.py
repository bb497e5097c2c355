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


def test_every_bench_operator_class_has_a_smoother_set():
    """The mixed-batch and serving legs draw their smoother sets from the
    package's operator table: every class they use has a stored file, cut or
    extended to the class's levels."""
    from paper_2603_01064_gb300.weights import operator_weights
    for n in bench.MIXED["sizes"]:
        for sg in bench.MIXED["sigmas"]:
            for al in bench.MIXED["alphas"]:
                L = n.bit_length() - 3  # log2(n) - 2
                assert len(operator_weights(sg, al, L)) == L - 1
    for n, L, sg, W in bench.serving_classes():
        assert len(W) == L - 1 and L == n.bit_length() - 3


def test_issued_mma_work_per_pixel():
    """Issued MMA flops per output pixel of the hidden convs: 6 products for
    three bf16 terms, 3 for the pair forms, 1 for one bf16; the form with
    three terms on the finest level only weights the two by pixels."""
    alg = bench.FLOPS_PER_PX["cnn_hidden"]
    assert bench.mma_flops_per_px("bf16_refine", "cnn_hidden", 512, 7) == 6 * alg
    assert bench.mma_flops_per_px("bf16x3_refine", "cnn_hidden", 512, 7) == 3 * alg
    assert bench.mma_flops_per_px("fp16_refine", "cnn_hidden", 512, 7) == 3 * alg
    assert bench.mma_flops_per_px("bf16fast_refine", "cnn_hidden", 512, 7) == alg
    px = [(512 >> l) ** 2 for l in range(6)]
    f0 = px[0] / sum(px)
    top = bench.mma_flops_per_px("bf16top_refine", "cnn_hidden", 512, 7)
    assert abs(top - (6 * f0 + 3 * (1 - f0)) * alg) < 1e-6 * alg
