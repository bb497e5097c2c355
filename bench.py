#!/usr/bin/env python
"""Throughput of the neural multigrid solve: right-hand sides solved per
second to relative residual 1e-6, the bf16 refinement form batched against
the plain fp32 cycle one right-hand side at a time on the same GPU.

One step = one full solve of a batch of right-hand sides (every row of the
cycle: residual, norms, smoother, output filter, fused residual+restriction,
coarsest Cholesky solve, prolongation; the refinement form adds the
compensated outer residual and the fp64 update) from x^0 = 0 until every
right-hand side meets the tolerance.  Inputs are resident in HBM when the
timed region starts; L2 is flushed (a 256 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c3|c2]
                  [--precision bf16_refine|bf16fast_refine|fp16_refine|fp32]

Default workload (c3): 2D BTTB deblurring on a 512 x 512 grid, Gaussian PSF
sigma 4 px truncated at 4 sigma, alpha 1e-2, 7 levels, 64 right-hand sides
(plane waves + rectangles, blurred, 1% noise).  The same run sweeps alpha
over {1e-4, 1e-3, 1e-2, 1e-1} with that operator's trained smoothers
("alpha_sweep"), times the fp32 form batched, the fp32 form one
right-hand side per call (the plain fp32 single-RHS cycle) and the other
16-bit forms ("compare"), and the smaller 128 x 128 problem ("secondary").

Under torchrun each rank solves its own batch (different seeds, the same
sizes): weak scaling with no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import nmg_inputs as I  # noqa: E402

WEIGHTS = os.path.join(ROOT, "paper_2603_01064_gb300", "weights")
METRIC = "RHS solved/s to 1e-6 rel. residual (BF16+refine vs FP32 plain); p50/p99 latency"

WORKLOADS = {
    # 2D BTTB deblurring, 512x512, PSF sigma 4 px (truncated at 4 sigma), 7 levels,
    # 64 right-hand sides (8 plane waves + 2 rectangles, blurred, 1% noise);
    # headline alpha 1e-2, the sweep over the four alphas reported beside it
    "c3": dict(name="2d_bttb_512x512_sigma4_alpha1e-2_L7_batch64", n=512, levels=7, alpha=1e-2,
               sigma=4.0, batch=64, rhs="waves_rects", rhs_seed=1003,
               weights="c3_2d_n512_s4_a1e-2.npz",
               sweep=[(1e-4, "c3_2d_n512_s4_a1e-4.npz"), (1e-3, "c3_2d_n512_s4_a1e-3.npz"),
                      (1e-2, "c3_2d_n512_s4_a1e-2.npz"), (1e-1, "c3_2d_n512_s4_a1e-1.npz")]),
    # 2D BTTB deblurring, 128x128, PSF sigma 2 px (truncated at 4 sigma), alpha 1e-2,
    # 5 levels, 256 right-hand sides (ellipses + Gaussian random field, blurred, 1% noise)
    "c2": dict(name="2d_bttb_128x128_sigma2_alpha1e-2_L5_batch256", n=128, levels=5, alpha=1e-2,
               sigma=2.0, batch=256, rhs="ellipses_grf", rhs_seed=1002,
               weights="c2_2d_n128_s2_a1e-2.npz", fno_weights="c2f_2d_n128_s2_a1e-2_fno.npz"),
}
PRECISION_TEXT = {
    "bf16top_refine": "bf16 tensor-core smoother with three bf16 terms per operand (six products) "
                      "on the finest level and bf16 pairs (three products) on the coarser levels, "
                      "fp32 accumulation, fp32 cycle vectors, compensated-fp32 outer residual, "
                      "fp64 update and coarse solve",
    "bf16_refine": "bf16 tensor-core smoother, every operand three bf16 terms (six products per "
                   "product, fp32 accumulation), fp32 cycle vectors, compensated-fp32 outer "
                   "residual, fp64 update and coarse solve",
    "bf16x3_refine": "bf16 tensor-core smoother with hi+lo bf16 operand pairs (three products) and "
                     "fp32 accumulation, fp32 cycle vectors, compensated-fp32 outer residual, fp64 "
                     "update and coarse solve",
    "bf16fast_refine": "bf16 tensor-core smoother (one bf16 per operand, fp32 accumulation), fp32 "
                       "cycle vectors, compensated-fp32 outer residual, fp64 update and coarse solve",
    "fp16_refine": "fp16 tensor-core smoother with split hi+lo fp16 operands (power-of-two scaled "
                   "network) and fp32 accumulation, fp32 cycle vectors, compensated-fp32 outer "
                   "residual, fp64 update and coarse solve",
    "fp32": "fp32 throughout (SIMT smoother), fp64 coarse solve",
}
DTYPE = {"bf16_refine": "bf16x3+f32+f64", "bf16x3_refine": "bf16x2+f32+f64",
         "bf16top_refine": "bf16x3/bf16x2+f32+f64",
         "bf16fast_refine": "bf16+f32+f64",
         "fp16_refine": "f16x2+f32+f64", "fp32": "f32"}

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x fp32 lanes x FMA x max clock
FLOPS_PER_PX = {"cnn_hidden": 2 * 9 * 32 * 32, "cnn_first": 2 * 9 * 32, "cnn_last": 2 * 9 * 32}
# tensor-core MMA flops per pixel actually issued by the hidden layers, per bf16 form
# (the roofline's "achieved" uses the algorithmic flops above)
# DRAM bytes per output pixel of the hidden convs, mean of the two hidden
# layers, from one ncu capture of the level-0 launches of the current kernel
# version (summarised under profiles/: the three-term form at 512x512 with
# 16 RHS, the pair form at 128x128 with 64 RHS); None where no capture exists
HIDDEN_DRAM_B_PER_UNIT = {("bf16_refine", 512): 203.5, ("bf16x3_refine", 128): 109.9}
MMA_FLOPS_PER_PX = {
    # three-term form per tap and K half: a1 x N = 96 ([w1 | w2 | w3]), a2 x N = 64, a3 x N = 32
    "bf16_refine": {"cnn_hidden": 2 * 9 * 32 * (96 + 64 + 32)},
    # pair form per tap and K half: hi A x N = 64 ([w_hi | w_lo]) and lo A x N = 32 (w_hi)
    "bf16x3_refine": {"cnn_hidden": 2 * 9 * 32 * (64 + 32)},
    "bf16fast_refine": {"cnn_hidden": 2 * 9 * 32 * 32},
    "fp16_refine": {"cnn_hidden": 2 * 9 * 32 * (64 + 32)},
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def make_rhs(wl, batch, seed):
    if wl["rhs"] == "ellipses_grf":
        f, _ = I.rhs_2d_ellipses_grf(wl["n"], batch, seed, wl["sigma"])
    else:
        f, _ = I.rhs_2d_waves_rects(wl["n"], batch, seed, wl["sigma"])
    return f


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def reduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def rank_seed(wl, rank):
    """Each replica solves its own batch: the right-hand-side seed depends on the rank."""
    return wl["rhs_seed"] + 7919 * rank


def aggregate(batch_per_rank, world, steps, max_total_ms):
    """Whole-job throughput: right-hand sides of all ranks / slowest rank's time."""
    return batch_per_rank * world * steps / (max_total_ms / 1e3)


# ---------------------------------------------------------------------------
# the CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_cycle_time(wl, seed, ncycles):
    """Seconds per cycle of the FP64 oracle (Algorithm 4, one right-hand
    side of the workload, from x^0 = 0 as in the outer iteration of Section
    3.2), over `ncycles` cycles."""
    import oracle as O
    import paper_2603_01064_gb300 as nmg_pkg  # weights loader only (no library call)
    W = nmg_pkg.load_weights(os.path.join(WEIGHTS, wl["weights"]))
    H = O.build_hierarchy_2d(I.gaussian_taps(wl["sigma"]), wl["n"], wl["alpha"], wl["levels"])
    f = make_rhs(wl, 1, seed)
    x = None
    t0 = time.perf_counter()
    for _ in range(ncycles):
        x = O.nmgf(H, W, 0, x, f)
    return (time.perf_counter() - t0) / ncycles


def oracle_cycles_to_converge(wl):
    """Cycles the FP64 oracle takes to reach 1e-6 on the workload's first
    right-hand side, as stored by tests/golden/make_oracle_cycles.py (a
    script that runs only the oracle); None if not stored."""
    p = os.path.join(ROOT, "tests", "golden", "oracle_cycles.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(wl["name"])
    return None if e is None else int(e["cycles"])


def oracle_rate_sample(wl, seed, ncycles, threads=None):
    """Oracle right-hand sides per second on a bounded sample: `ncycles`
    cycles of one right-hand side timed, scaled by the oracle's own cycle
    count to 1e-6.  threads: run in a child process with every BLAS / OpenMP
    pool limited to that many threads (None: this process, all cores)."""
    if threads is None:
        t_cyc = oracle_cycle_time(wl, seed, ncycles)
    else:
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                  "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
            env[k] = str(threads)
        env.pop("RANK", None)
        env.pop("WORLD_SIZE", None)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-cycle-probe",
                            str(ncycles), "--workload", wl["key"], "--probe-seed", str(seed)],
                           capture_output=True, text=True, env=env, timeout=900)
        if r.returncode != 0:
            return None, None, None
        t_cyc = float(json.loads(r.stdout.strip().splitlines()[-1])["s_per_cycle"])
    cyc = oracle_cycles_to_converge(wl)
    if not cyc:
        return None, t_cyc, None
    return 1.0 / (t_cyc * cyc), t_cyc, cyc


REF_CYCLES_PER_STEP = 1


def run_reference(args, wl, world, rank):
    """The oracle timed on the host cores: each step is one cycle of one
    right-hand side of the workload (a bounded sample; a whole 512 x 512
    solve takes minutes on the CPU), and right-hand sides per second are
    that cycle time times the oracle's own cycle count to 1e-6."""
    if rank != 0:
        return
    cores = os.cpu_count()
    cyc = oracle_cycles_to_converge(wl)
    for k in range(args.warmup):
        oracle_cycle_time(wl, wl["rhs_seed"], REF_CYCLES_PER_STEP)
    times = []
    for k in range(args.steps):
        times.append(oracle_cycle_time(wl, wl["rhs_seed"], REF_CYCLES_PER_STEP)
                     * REF_CYCLES_PER_STEP)
    t_cyc = sum(times) / (args.steps * REF_CYCLES_PER_STEP)
    value = 1.0 / (t_cyc * cyc) if cyc else None
    sample = (f"{REF_CYCLES_PER_STEP} cycle of 1 right-hand side of the workload per step "
              f"(FP64 numpy oracle, BLAS threads = all host cores); RHS/s = 1 / (seconds per "
              f"cycle x {cyc} cycles, the oracle's own count to 1e-6 on this workload)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "n": wl["n"], "levels": wl["levels"],
                       "batch": 1, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our CUDA path
# ---------------------------------------------------------------------------

def timed_steps(stepfn, K, flush, stream):
    """CUDA events on the library's stream around each of K steps, L2
    written over (256 MiB) before each; returns (ms list, step results)."""
    import torch
    times, res = [], []
    for k in range(K):
        flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res.append(stepfn())
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times, res


def solve_summary(B, tp, rp):
    return {"value": B * len(tp) / (sum(tp) / 1e3), "unit": "RHS/s", "batch": B,
            "mean_cycles": float(np.mean([r[0].mean() for r in rp])),
            "max_cycles": int(max(r[0].max() for r in rp)),
            "converged": int(min((r[1] == 0).sum() for r in rp)),
            "max_relres": float(max(r[2].max() for r in rp))}


def mma_flops_per_px(prec, dom, n, levels):
    """Issued MMA flops per output pixel of a kernel class; for the form with
    three terms on the finest level and pairs below, the pixel-weighted mean
    over the smoother levels."""
    if prec == "bf16top_refine":
        px = [(n >> l) ** 2 for l in range(levels - 1)]
        f0 = px[0] / sum(px)
        return (f0 * MMA_FLOPS_PER_PX["bf16_refine"][dom] +
                (1 - f0) * MMA_FLOPS_PER_PX["bf16x3_refine"][dom])
    return MMA_FLOPS_PER_PX[prec][dom]


def roofline_of(kern, prec, n, levels, peaks, peak_src):
    """Roofline of the dominant kernel class: algorithmic work per unit x
    units / the class's summed CUDA-event time."""
    dom = max(kern, key=lambda k: kern[k]["ms"])
    d = kern[dom]
    refine = prec != "fp32"
    if dom in FLOPS_PER_PX and refine:
        fl = FLOPS_PER_PX[dom]
        achieved = fl * d["units"] / (d["ms"] / 1e3) / 1e12
        mpx = mma_flops_per_px(prec, dom, n, levels)
        issued = mpx * d["units"] / (d["ms"] / 1e3) / 1e12
        peak = peaks["bf16_tflops_sustained"]
        bpu = HIDDEN_DRAM_B_PER_UNIT.get((prec, n)) if dom == "cnn_hidden" else None
        traffic = bpu * d["units"] / d["launches"] if bpu else None
        return {"kernel": f"{dom} (tcgen05 bf16 3x3 conv)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_bytes_per_unit": bpu,
                "traffic_source": (f"ncu dram__bytes_read+write of the {n}x{n} level, scaled to "
                                   "this launch's units") if bpu else None,
                "peak_source": f"{peak_src} bf16_tflops_sustained",
                "flop_per_unit": fl, "unit_def": "output pixel x active right-hand side",
                "mma_issued_tflops": issued,
                "mma_issued_flop_per_unit": mpx,
                "launch_ms": d["ms"] / d["launches"]}
    if dom in FLOPS_PER_PX:
        achieved = FLOPS_PER_PX[dom] * d["units"] / (d["ms"] / 1e3) / 1e12
        return {"kernel": f"{dom} (fp32 SIMT 3x3 conv)", "bound": "alu", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": None,
                "peak_source": "152 SMs x 128 fp32 lanes x 2 flop x 2070 MHz (derived)",
                "flop_per_unit": FLOPS_PER_PX[dom], "launch_ms": d["ms"] / d["launches"]}
    bpu = {"residual": 12, "restrict": 9, "prolong": 9, "filter": 8,
           "refine_residual": 16}.get(dom, 8)
    achieved = bpu * d["units"] / (d["ms"] / 1e3) / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
            "peak_source": peak_src, "bytes_per_unit": bpu,
            "launch_ms": d["ms"] / d["launches"]}


def kernel_breakdown(kern, prec, steps, peaks):
    prof_total = sum(v["ms"] for v in kern.values())
    breakdown = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / steps,
                     "share": v["ms"] / prof_total} for k, v in kern.items()}
    # the memory-bound classes against the measured HBM copy bandwidth:
    # algorithmic bytes per unit (grid point x active right-hand side, every
    # level of the class together) / class time
    act_b = {"bf16_refine": 192, "bf16x3_refine": 128, "fp16_refine": 128, "bf16fast_refine": 64,
             "fp32": 128}[prec]
    hbm_bpu = {"restrict": 9, "refine_residual": 16,
               "prolong": 9, "filter": 8, "cnn_first": 4 + act_b, "cnn_last": 40}
    if prec == "fp32":
        hbm_bpu.pop("cnn_first")
        hbm_bpu.pop("cnn_last")
    for k, bpu_k in hbm_bpu.items():
        if k in kern and kern[k]["ms"] > 0:
            gbs = bpu_k * kern[k]["units"] / (kern[k]["ms"] / 1e3) / 1e9
            breakdown[k].update({"bytes_per_unit": bpu_k, "achieved_gbs": gbs,
                                 "hbm_frac": gbs / peaks["hbm_gbs"]})
    return breakdown


def run_ours(args, wl, world, rank, local):
    import torch
    import paper_2603_01064_gb300 as nmg

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = nmg.Context(local, stream=stream.cuda_stream)
    if args.no_graphs:
        ctx.set_graphs(False)
    W = nmg.load_weights(os.path.join(WEIGHTS, wl["weights"]))
    taps = I.gaussian_taps(wl["sigma"])
    prec = args.precision

    def hier(p, alpha=None, Wx=None):
        return nmg.Hierarchy(ctx, dim=2, n=wl["n"], levels=wl["levels"],
                             alpha=wl["alpha"] if alpha is None else alpha,
                             taps=taps, precision=p, weights=W if Wx is None else Wx)

    G = hier(prec)
    B = args.batch or wl["batch"]
    # launch shapes per level, timed on this GPU (outside the timed region);
    # with --tune-cache the choices are read from / appended to that file, so
    # that a profiled run (whose timings ncu distorts) launches the shapes the
    # plain run chose
    G.autotune(B, args.tune_cache)
    f_np = make_rhs(wl, B, rank_seed(wl, rank))
    refine = prec != "fp32"
    udt = torch.float64 if refine else torch.float32
    f = torch.tensor(f_np, dtype=torch.float32, device="cuda")
    u = torch.zeros(f.shape, dtype=udt, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(Gx=G, fx=f, ux=u, max_cycles=100):
        ux.zero_()
        return Gx.solve(fx, ux, rtol=1e-6, max_cycles=max_cycles)

    if args.ncu:
        # one solve only: the command profiled by ncu
        cyc, st, rr = step()
        torch.cuda.synchronize()
        print(json.dumps({"ncu_run": wl["name"], "precision": prec, "batch": B,
                          "cycles": float(cyc.mean()), "max_relres": float(rr.max()),
                          "launches": ctx.launches()}))
        return
    for _ in range(max(args.warmup, 0)):
        cyc, st, rr = step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    l0 = ctx.launches()
    barrier(world)
    torch.cuda.synchronize()
    times, res = timed_steps(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = ctx.launches() - l0
    clk = clocks.stop()
    total_ms = reduce_max(sum(times), world)
    value = aggregate(B, world, args.steps, total_ms)
    converged = bool(all((r[1] == 0).all() for r in res))
    max_relres = float(max(r[2].max() for r in res))
    mean_cycles = float(np.mean([r[0].mean() for r in res]))

    # ---- per-kernel timing with CUDA events on the library's stream (same steps again)
    ksteps = max(1, min(args.steps, 3))
    ctx.profile(True)
    timed_steps(step, ksteps, flush, stream)
    ctx.profile(False)
    kern = {}
    for kind, name in enumerate(nmg.KERNEL_CLASSES):
        c, ms, units = ctx.profile_read(kind)
        if c:
            kern[name] = {"launches": c, "ms": ms, "units": units}
    peaks, peak_src = load_peaks()
    roof = roofline_of(kern, prec, wl["n"], wl["levels"], peaks, peak_src)
    breakdown = kernel_breakdown(kern, prec, ksteps, peaks)

    # ---- the comparison forms on the same GPU and right-hand sides
    compare = {}
    if not args.no_compare:
        for p in ["fp32", "bf16fast_refine", "bf16x3_refine", "bf16_refine", "bf16top_refine",
                  "fp16_refine"]:
            if p == prec:
                continue
            Gp = hier(p)
            Gp.autotune(B)
            up = torch.zeros(f.shape, dtype=torch.float32 if p == "fp32" else torch.float64,
                             device="cuda")
            step_p = (lambda Gp=Gp, up=up: step(Gp, f, up))
            step_p()
            tp, rp = timed_steps(step_p, max(1, min(args.steps, 2)), flush, stream)
            compare[p + "_batched"] = solve_summary(B, tp, rp)
            Gp.close()
            del up
        # plain fp32 single-RHS cycle: one right-hand side per solve call
        Gs = hier("fp32")
        nsingle = min(16, B)
        us = torch.zeros((1, wl["n"], wl["n"]), dtype=torch.float32, device="cuda")
        step(Gs, f[0:1], us)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rr1, cc1 = [], []
        for i in range(nsingle):
            r1 = step(Gs, f[i:i + 1], us)
            rr1.append(r1[2][0])
            cc1.append(r1[0][0])
        e1.record(stream)
        e1.synchronize()
        compare["fp32_single_rhs"] = {
            "value": nsingle / (e0.elapsed_time(e1) / 1e3), "unit": "RHS/s", "batch": 1,
            "rhs_timed": nsingle, "mean_cycles": float(np.mean(cc1)),
            "max_relres": float(max(rr1))}
        Gs.close()
        compare["headline_vs_fp32_single_rhs"] = value / world / compare["fp32_single_rhs"]["value"]

    # ---- the paper's classical comparators on the same operator and right-hand sides
    classical = None
    if not args.no_classical:
        classical = classical_leg(ctx, wl, f, taps, stream, mean_cycles)

    # ---- alpha sweep of the workload's operator (its own trained smoothers per alpha)
    sweep = None
    if wl.get("sweep") and not args.no_sweep:
        sweep = sweep_leg(ctx, wl, f, taps, flush, stream, rank)

    # ---- end to end through the C ABI with host buffers (pinned): f copied
    # in, the solve from the zero initial guess, u copied back, every step
    fh = torch.tensor(f_np, dtype=torch.float32).pin_memory().numpy()
    uh = torch.zeros(f.shape, dtype=udt).pin_memory().numpy()
    G.solve_host(fh, uh, zero_start=True)  # warm the staging buffers
    barrier(world)
    t0 = time.perf_counter()
    for k in range(args.steps):
        G.solve_host(fh, uh, zero_start=True)
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e = {"value": B * world * args.steps / e2e_s, "unit": "RHS/s",
           "h2d_bytes_per_step": int(fh.nbytes), "d2h_bytes_per_step": int(uh.nbytes),
           "call": "nmg_solve_host_zero"}
    G.close()
    del u, f

    # ---- the smaller 128x128 problem as a secondary line
    secondary = None
    if wl["key"] != "c2" and not args.no_secondary:
        secondary = secondary_leg(ctx, WORKLOADS["c2"], prec, flush, stream, rank)

    # ---- serving: a Poisson stream of mixed-size requests through the
    # continuous-batching server (p50/p99 latency beside throughput)
    serving = None
    if not args.no_serving:
        serving = serving_leg(ctx, rank)
    # ---- mixed batch: 24 operator classes in one multi-solve
    mixed = None
    if not args.no_mixed:
        mixed = mixed_leg(ctx, flush, stream, rank)
    fno = None
    if not args.no_fno:
        fno = fno_leg(ctx, WORKLOADS["c2"])
    hbm = None
    if not args.no_hbm_apply:
        hbm = hbm_apply_leg(ctx, flush, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ncyc = 2
        rate, t_cyc, ocyc = oracle_rate_sample(wl, wl["rhs_seed"], ncyc)
        rate1, t_cyc1, _ = oracle_rate_sample(wl, wl["rhs_seed"], 1, threads=1)
        cpu = {"value": rate, "unit": "RHS/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"{ncyc} cycles of 1 right-hand side of the workload timed "
                          f"({t_cyc:.2f} s per cycle, numpy FP64, BLAS threads = all host "
                          f"cores), scaled by the oracle's own {ocyc} cycles to 1e-6"),
               "one_core": {"value": rate1, "unit": "RHS/s", "cores": 1,
                            "s_per_cycle": t_cyc1,
                            "sample": "1 cycle of 1 right-hand side, every BLAS / OpenMP pool "
                                      "limited to 1 thread, same scaling"}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec],
                "data": "synthetic",
                "config": {"workload": wl["name"], "n": wl["n"], "levels": wl["levels"],
                           "sigma_px": wl["sigma"], "alpha": wl["alpha"],
                           "batch_per_gpu": B, "precision": prec,
                           "precision_detail": PRECISION_TEXT[prec],
                           "l2": "flushed (256 MiB write) before every timed step",
                           "parallelism": f"replicas x{world}"},
                "converged": converged, "max_relres": max_relres, "mean_cycles": mean_cycles,
                "compare": compare, "classical": classical, "alpha_sweep": sweep,
                "mixed_batch": mixed, "roofline": roof,
                "kernels": breakdown, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
                "secondary": secondary, "serving": serving, "fno_smoother": fno,
                "hbm_apply": hbm}
        print(json.dumps(line), flush=True)


CLASSICAL_RHS = 16  # right-hand sides of the workload the classical comparators solve


def classical_leg(ctx, wl, f, taps, stream, neural_cycles):
    """The comparators of the paper's tables on the workload's operator, fp32,
    to the same 1e-6: the backslash V-cycle of Algorithm 1 with weighted
    Jacobi smoothing (nu1 = 5, nu2 = 0) and conjugate gradients, on the
    first CLASSICAL_RHS right-hand sides (one solve call each form, CUDA
    events around it), beside the neural cycle's count."""
    import torch
    import paper_2603_01064_gb300 as nmg
    B = min(CLASSICAL_RHS, f.shape[0])
    G = nmg.Hierarchy(ctx, dim=2, n=wl["n"], levels=wl["levels"], alpha=wl["alpha"], taps=taps,
                      precision="fp32", weights=nmg.load_weights(os.path.join(WEIGHTS, wl["weights"])))
    fs = f[:B].contiguous()
    out = {"rhs": B, "precision": "fp32", "neural_mean_cycles": neural_cycles}
    for name, fn in [("mg_jacobi_nu1_5", lambda u: G.solve_mg_jacobi(fs, u, 1e-6, 20000, 5, 0)),
                     ("cg", lambda u: G.solve_cg(fs, u, 1e-6, 20000))]:
        u = torch.zeros_like(fs)
        fn(u)  # warm-up (graph capture)
        u.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cyc, st, rr = fn(u)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"value": B / (ms / 1e3), "unit": "RHS/s", "mean_cycles": float(np.mean(cyc)),
                     "max_cycles": int(np.max(cyc)), "converged": int((st == 0).sum()),
                     "max_relres": float(np.max(rr)), "ms": ms}
    G.close()
    return out


SWEEP_ORACLE_SAMPLE = 1  # right-hand sides per alpha checked against the oracle's cycle


# the CNN smoothers of the alpha = 1e-3 operator take about 50 cycles to
# 1e-6, those of alpha = 1e-4 about 300; the limit leaves them room
SWEEP_MAX_CYCLES = 400


def sweep_leg(ctx, wl, f, taps, flush, stream, rank):
    """For each alpha of the workload's sweep, with that operator's trained
    CNN smoothers: a bf16 split refinement solve of the whole batch to 1e-6
    (at most SWEEP_MAX_CYCLES cycles), its cycles and residuals, the final residual of
    sampled right-hand sides recomputed by the FP64 oracle's own apply, and
    one cycle from zero of the whole batch against the oracle's cycle for a
    sampled right-hand side (the per-cycle parity bar of the bf16 form is
    1e-3, element-wise error reported beside the norm-wise one)."""
    import torch
    import oracle as O
    import paper_2603_01064_gb300 as nmg
    B = f.shape[0]
    out = []
    for alpha, wname in wl["sweep"]:
        Wa = nmg.load_weights(os.path.join(WEIGHTS, wname))
        G = nmg.Hierarchy(ctx, dim=2, n=wl["n"], levels=wl["levels"], alpha=alpha, taps=taps,
                          precision="bf16_refine", weights=Wa)
        G.autotune(B)
        u = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
        G.solve(f, u, rtol=1e-6, max_cycles=SWEEP_MAX_CYCLES)
        tp, rp = timed_steps(lambda: (u.zero_(), G.solve(f, u, rtol=1e-6,
                                                         max_cycles=SWEEP_MAX_CYCLES))[1],
                             1, flush, stream)
        row = {"alpha": alpha, "weights": wname, **solve_summary(B, tp, rp)}
        if rank == 0:
            H = O.build_hierarchy_2d(taps, wl["n"], alpha, wl["levels"])
            idx = [0, B - 1][:max(1, min(2, B))]
            fs = f[idx].double().cpu().numpy()
            row["oracle_relres_sampled"] = [float(v) for v in
                                            O.relres(H, fs, u[idx].cpu().numpy())]
            u.zero_()
            G.cycle(f, u)
            torch.cuda.synchronize()
            k = idx[:SWEEP_ORACLE_SAMPLE]
            ref = O.nmgf(H, Wa, 0, None, f[k].double().cpu().numpy())
            got = u[k].cpu().numpy()
            d = (got - ref).reshape(len(k), -1)
            rf = ref.reshape(len(k), -1)
            row["one_cycle_vs_oracle"] = {
                "rhs": k,
                "normwise": float(np.max(np.linalg.norm(d, axis=1) / np.linalg.norm(rf, axis=1))),
                "elementwise": float(np.max(np.abs(d).max(axis=1) / np.abs(rf).max(axis=1))),
                "bar": 1e-3}
        out.append(row)
        G.close()
        del u
    return out


def secondary_leg(ctx, wl, prec, flush, stream, rank):
    """The 128 x 128 problem (sigma 2 px, alpha 1e-2, 5 levels, 256
    right-hand sides): the same form batched and the plain fp32 cycle one
    right-hand side per call."""
    import torch
    import paper_2603_01064_gb300 as nmg
    W = nmg.load_weights(os.path.join(WEIGHTS, wl["weights"]))
    taps = I.gaussian_taps(wl["sigma"])
    B = wl["batch"]
    f = torch.tensor(make_rhs(wl, B, rank_seed(wl, rank)), dtype=torch.float32, device="cuda")
    out = {"workload": wl["name"]}
    for p in [prec, "fp32"]:
        G = nmg.Hierarchy(ctx, dim=2, n=wl["n"], levels=wl["levels"], alpha=wl["alpha"],
                          taps=taps, precision=p, weights=W)
        G.autotune(B)
        u = torch.zeros(f.shape, dtype=torch.float32 if p == "fp32" else torch.float64,
                        device="cuda")
        step = (lambda G=G, u=u: (u.zero_(), G.solve(f, u, rtol=1e-6, max_cycles=100))[1])
        step()
        tp, rp = timed_steps(step, 3, flush, stream)
        out[p + "_batched"] = solve_summary(B, tp, rp)
        if p == "fp32":
            us = torch.zeros((1, wl["n"], wl["n"]), dtype=torch.float32, device="cuda")
            G.solve(f[0:1], us)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(16):
                us.zero_()
                G.solve(f[i:i + 1], us)
            out["fp32_single_rhs"] = {"value": 16 / (time.perf_counter() - t0), "unit": "RHS/s",
                                      "batch": 1, "rhs_timed": 16}
        G.close()
    return out


def operator_weights(sigma, alpha, levels):
    from paper_2603_01064_gb300.weights import operator_weights as ow
    return ow(sigma, alpha, levels)


# Mixed batch: 512 right-hand sides drawn uniformly (seeded) over 24
# operator classes, grid sides {64, 128, 256, 512} x PSF sigma {1, 2, 4} px x
# alpha {1e-3, 1e-2}, levels log2(n) - 2 (coarsest 8 x 8); one
# nmg_solve_multi call: one captured graph per outer iteration with the
# classes as parallel branches, launch shapes autotuned per class
MIXED = dict(rhs=512, seed=777, sizes=[64, 128, 256, 512], sigmas=[1.0, 2.0, 4.0],
             alphas=[1e-3, 1e-2], max_cycles=250, steps=2)


def mixed_leg(ctx, flush, stream, rank):
    """The mixed batch solved to 1e-6 in one multi-solve (CUDA events around
    each of MIXED['steps'] solves after one untimed one), beside the same
    classes solved one after another with nmg_solve; per class its cycles
    and convergence; kernels launched per outer iteration."""
    import torch
    import paper_2603_01064_gb300 as nmg
    classes = [(n, sg, al) for n in MIXED["sizes"] for sg in MIXED["sigmas"]
               for al in MIXED["alphas"]]
    rng = np.random.default_rng(MIXED["seed"] + 7919 * rank)
    counts = np.bincount(rng.integers(0, len(classes), MIXED["rhs"]), minlength=len(classes))
    items, meta = [], []
    for k, ((n, sg, al), B) in enumerate(zip(classes, counts)):
        if B == 0:
            continue
        L = int(np.log2(n)) - 2
        G = nmg.Hierarchy(ctx, dim=2, n=n, levels=L, alpha=al, taps=I.gaussian_taps(sg),
                          precision="bf16_refine", weights=operator_weights(sg, al, L))
        G.autotune(int(B))
        f, _ = I.rhs_2d_waves_rects(n, int(B), MIXED["seed"] + 31 * k + 7919 * rank, sg)
        fd = torch.tensor(f, dtype=torch.float32, device="cuda")
        items.append((G, fd, torch.zeros(fd.shape, dtype=torch.float64, device="cuda")))
        meta.append({"n": n, "sigma_px": sg, "alpha": al, "levels": L, "rhs": int(B)})

    def multi():
        for _, _, u in items:
            u.zero_()
        return nmg.solve_multi(ctx, items, rtol=1e-6, max_cycles=MIXED["max_cycles"])

    multi()
    torch.cuda.synchronize()
    l0 = ctx.launches()
    tp, rp = timed_steps(multi, MIXED["steps"], flush, stream)
    kernels = (ctx.launches() - l0) / MIXED["steps"]
    iters = max(int(r[0].max()) for r in rp[-1]) + 1

    def sequential():
        out = []
        for G, f, u in items:
            u.zero_()
            out.append(G.solve(f, u, rtol=1e-6, max_cycles=MIXED["max_cycles"]))
        return out

    sequential()
    ts, _ = timed_steps(sequential, 1, flush, stream)
    total = int(sum(m["rhs"] for m in meta))
    per_class = []
    for m, r in zip(meta, rp[-1]):
        per_class.append(dict(m, mean_cycles=float(r[0].mean()), max_cycles=int(r[0].max()),
                              converged=int((r[1] == 0).sum()), max_relres=float(r[2].max())))
    for G, _, _ in items:
        G.close()
    return {"rhs": total, "classes": len(meta), "precision": "bf16_refine",
            "value": total * len(tp) / (sum(tp) / 1e3), "unit": "RHS/s",
            "ms_per_solve": float(np.mean(tp)), "outer_iterations": iters,
            "graph_launches_per_iteration": 1 if ctx.graphs else None,
            "kernels_per_iteration": kernels / iters,
            "converged": int(sum(c["converged"] for c in per_class)),
            "sequential_value": total / (ts[0] / 1e3),
            "note": "one nmg_solve_multi call; sequential_value: the same classes solved one "
                    "nmg_solve call after another",
            "per_class": per_class}


# Serving: grid sides n = 2^e with e uniform in {6..11} (log-uniform 64^2 ..
# 2048^2), levels e - 2 (coarsest 8 x 8), PSF sigma = max(1, 8 n / 2048) px,
# alpha 1e-3 (the 2048^2 class: 9 levels, sigma 8 px).  Smoother sets per
# sigma (trained level-wise for that sigma and alpha); a class with more
# smoother levels than its set repeats the set's last (coarsest) net.
SERVING = dict(requests=240, burst=60, load=0.8, seed=4242, alpha=1e-3, max_cycles=300,
               exps=[6, 7, 8, 9, 10, 11],
               slots={6: 64, 7: 64, 8: 32, 9: 16, 10: 8, 11: 4}, fp32_sample=12)


def serving_classes():
    """(n, levels, sigma, weights) of the serving size classes."""
    out = []
    for e in SERVING["exps"]:
        n = 1 << e
        sigma = max(1.0, 8.0 * n / 2048.0)
        L = e - 2
        out.append((n, L, sigma, operator_weights(sigma, SERVING["alpha"], L)))
    return out


FNO = dict(width=64, layers=4, modes=8, ksize=3, seed=0, reps=5)


def fno_leg(ctx, wl):
    """The FNO smoother of Appendix A (the paper's 2D hyperparameters at
    h = 1/128: 64 channels, 4 Fourier layers, 3x3 W term; 8 retained modes
    per axis, the most a 16x16 coarsest smoother level holds) applied once to
    the fine level of the workload's whole batch in fp32, with seeded random
    weights (its cost does not depend on the weights).  CUDA events around
    `reps` applications after one warm-up; flops counted per output pixel:
    lift and projection 4c, per layer 2 c^2 k^2 (W term) + 8 c m (the
    truncated DFTs' row passes) + the smaller column passes and mode mixing."""
    import torch
    import paper_2603_01064_gb300 as nmg
    n, L, B = wl["n"], wl["levels"], wl["batch"]
    taps = I.gaussian_taps(wl["sigma"])
    c, nl, m, k = FNO["width"], FNO["layers"], FNO["modes"], FNO["ksize"]
    W = I.random_fno_weights(L - 1, FNO["seed"], width=c, layers=nl, modes=m, ksize=k)
    G = nmg.Hierarchy(ctx, dim=2, n=n, levels=L, alpha=wl["alpha"], taps=taps, precision="fp32",
                      weights=W)
    b = torch.tensor(make_rhs(wl, B, 99), dtype=torch.float32, device="cuda")
    h = torch.empty_like(b)
    G.smooth(0, b, h)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(FNO["reps"]):
        G.smooth(0, b, h)
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / FNO["reps"]
    G.close()
    per_px = (4 * c + nl * (2 * c * c * k * k + 8 * c * m) +
              nl * (32 * m * m * c / n + 16 * m * m * c * c / (n * n)))
    tflops = per_px * n * n * B / (ms / 1e3) / 1e12
    return {"config": {"n": n, "batch": B, "width": c, "layers": nl, "modes": m, "ksize": k,
                       "precision": "fp32", "weights": "seeded random"},
            "ms_per_application": ms, "flop_per_pixel": per_px, "achieved_tflops": tflops,
            "bound": "alu", "peak_tflops": FP32_PEAK_TFLOPS,
            "frac": tflops / FP32_PEAK_TFLOPS,
            "peak_source": "152 SMs x 128 fp32 lanes x 2 flop x 2070 MHz (derived)"}


HBM_APPLY = dict(reps=5, ops=[  # (n, levels, sigma px, alpha, weights, batch)
    (128, 5, 2.0, 1e-2, "c2_2d_n128_s2_a1e-2.npz", 2048),
    (512, 7, 4.0, 1e-2, "c3_2d_n512_s4_a1e-2.npz", 128)])


def hbm_apply_leg(ctx, flush, stream):
    """The fine-level operator kernels on vectors larger than L2 (134 MB per
    fp32 vector; L2 written over before every launch): the residual
    r = y - A x (12 B per grid point: x, y in, r out), the fused residual +
    full-weighting restriction (9 B: x, y in, a quarter-size vector out) and
    the prolongation + correction x += P e (9 B: x in and out, e a quarter).
    CUDA events around each launch on the library's stream; GB/s from the
    algorithmic bytes, against the measured HBM copy bandwidth."""
    import torch
    import paper_2603_01064_gb300 as nmg
    peaks, src = load_peaks()
    out = []
    for n, L, sg, al, wname, B in HBM_APPLY["ops"]:
        Wx = nmg.load_weights(os.path.join(WEIGHTS, wname))
        G = nmg.Hierarchy(ctx, dim=2, n=n, levels=L, alpha=al, taps=I.gaussian_taps(sg),
                          precision="fp32", weights=Wx)
        G.autotune(B)
        g = torch.Generator(device="cuda").manual_seed(5)
        x = torch.randn((B, n, n), device="cuda", generator=g)
        y = torch.randn((B, n, n), device="cuda", generator=g)
        r = torch.empty_like(x)
        yc = torch.empty((B, n // 2, n // 2), device="cuda")
        ops = {"residual": (lambda: G.residual(0, x, y, r), 12),
               "residual_restrict": (lambda: G.residual_restrict(0, x, y, yc), 9),
               "prolong_correct": (lambda: G.prolong_correct(0, yc, r), 9)}
        row = {"operator": f"{n}x{n} sigma {sg:g} px alpha {al:g}", "batch": B,
               "vector_mb": B * n * n * 4 / 1e6}
        for name, (fn, bpp) in ops.items():
            fn()
            torch.cuda.synchronize()
            tot = 0.0
            for k in range(HBM_APPLY["reps"]):
                flush.fill_(k & 0xFF)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            ms = tot / HBM_APPLY["reps"]
            gbs = bpp * B * n * n / (ms / 1e3) / 1e9
            row[name] = {"ms": ms, "bytes_per_unit": bpp, "achieved_gbs": gbs,
                         "hbm_frac": gbs / peaks["hbm_gbs"]}
        G.close()
        del x, y, r, yc
        out.append(row)
    return {"peak_gbs": peaks["hbm_gbs"], "peak_source": src, "results": out}


def serving_leg(ctx, rank):
    """Continuous batching over the serving size classes (bf16 refinement
    form, every request to 1e-6 or the cycle limit), all hierarchies
    resident, pools admitted by free device memory:
      1. saturation: SERVING['burst'] requests submitted at once; completed
         requests per second = the saturated throughput X;
      2. a seeded Poisson stream of SERVING['requests'] requests at rate
         load x X in real time: throughput and p50 / p99 latency (completion
         - submission, host clock);
      3. the plain fp32 cycle one request at a time (no batching, no queue)
         on a sample of the same requests: requests per second and the
         per-request latencies."""
    import torch
    import paper_2603_01064_gb300 as nmg
    from paper_2603_01064_gb300 import serve
    cls = serving_classes()
    ops = [serve.Operator(n, L, sg, SERVING["alpha"], W, "bf16_refine",
                          SERVING["slots"][int(np.log2(n))]) for (n, L, sg, W) in cls]
    srv, hs, ids = serve.build_server(ctx, ops, budget_bytes=0,
                                      max_cycles=SERVING["max_cycles"])
    seed = SERVING["seed"] + 7919 * rank
    burst = serve.poisson_stream(ops, SERVING["burst"], 1e9, seed + 1, rhs_batch=4)
    t_b, done_b = serve.run_stream(srv, ids, burst, time_limit_s=120.0)
    sat = len(done_b) / t_b if t_b > 0 else None
    rate = SERVING["load"] * sat if sat else 10.0
    reqs = serve.poisson_stream(ops, SERVING["requests"], rate, seed, rhs_batch=4)
    elapsed, done = serve.run_stream(srv, ids, reqs, time_limit_s=120.0)
    lat = serve.latency_stats(done)
    per_class = {}
    for k, o in enumerate(ops):
        dk = [r for r in done if r.op == k]
        if dk:
            per_class[str(o.n)] = {"requests": len(dk),
                                   "mean_cycles": float(np.mean([r.info[0] for r in dk])),
                                   "converged": int(sum(r.info[1] == 0 for r in dk)),
                                   **serve.latency_stats(dk)}
    out = {"requests": len(reqs), "completed": len(done), "wall_s": elapsed,
           "saturated_rhs_s": sat, "rate_rps": rate, "load": SERVING["load"],
           "throughput_rhs_s": len(done) / elapsed if elapsed > 0 else None,
           "converged": int(sum(r.info and r.info[1] == 0 for r in done)),
           "sizes": [o.n for o in ops], "sigma_px": [o.sigma for o in ops], "alpha": SERVING["alpha"],
           "max_slots": [o.slots for o in ops], "precision": "bf16_refine",
           "admission": "free device memory (pools grow on demand)", **lat, "per_class": per_class}
    srv.close()
    for G in hs:
        G.close()
    # the plain fp32 cycle, one request at a time, on a sample of the stream
    sample = reqs[:SERVING["fp32_sample"]]
    hs32 = {}
    lat32, cyc32, conv32 = [], [], 0
    t0 = time.perf_counter()
    for r in sample:
        o = ops[r.op]
        if r.op not in hs32:
            hs32[r.op] = nmg.Hierarchy(ctx, dim=2, n=o.n, levels=o.levels, alpha=o.alpha,
                                       taps=I.gaussian_taps(o.sigma), precision="fp32",
                                       weights=o.weights)
        G = hs32[r.op]
        ts = time.perf_counter()
        fd = torch.tensor(r.f[None], device="cuda")
        ud = torch.zeros_like(fd)
        cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=SERVING["max_cycles"])
        ud.cpu()
        lat32.append(time.perf_counter() - ts)
        cyc32.append(int(cyc[0]))
        conv32 += int(st[0] == 0)
    t32 = time.perf_counter() - t0
    out["fp32_one_at_a_time"] = {
        "requests": len(sample), "value": len(sample) / t32, "unit": "RHS/s",
        "p50_ms": 1e3 * float(np.percentile(lat32, 50)), "p99_ms": 1e3 * float(np.percentile(lat32, 99)),
        "mean_cycles": float(np.mean(cyc32)), "converged": conv32,
        "note": "solve time per request alone (setup of the hierarchies excluded)"}
    for G in hs32.values():
        G.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=0, help="override the batch (profiling runs)")
    ap.add_argument("--ncu", action="store_true", help="a single solve, nothing else (profiling)")
    ap.add_argument("--tune-cache", default=None,
                    help="launch-shape choices file (read if present, else written)")
    ap.add_argument("--precision", default="bf16_refine", choices=sorted(PRECISION_TEXT))
    ap.add_argument("--no-compare", action="store_true", help="skip the comparison forms")
    ap.add_argument("--no-sweep", action="store_true", help="skip the alpha sweep")
    ap.add_argument("--no-classical", action="store_true",
                    help="skip the classical comparators (Jacobi V-cycle, CG)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 128x128 line")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the 24-class mixed batch (one multi-solve)")
    ap.add_argument("--no-fno", action="store_true", help="skip the FNO smoother timing")
    ap.add_argument("--no-hbm-apply", action="store_true",
                    help="skip the out-of-L2 operator apply timing")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel eagerly instead of replaying captured iterations "
                         "(profiler launch lists)")
    ap.add_argument("--oracle-cycle-probe", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--probe-seed", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload], key=args.workload)
    if args.oracle_cycle_probe:
        # child process of the one-core CPU baseline (thread pools set by the parent)
        t = oracle_cycle_time(wl, args.probe_seed, args.oracle_cycle_probe)
        print(json.dumps({"s_per_cycle": t}))
        return
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, wl, world, rank)
    else:
        run_ours(args, wl, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
