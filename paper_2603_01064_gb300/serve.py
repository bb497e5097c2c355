"""Serving driver: a seeded Poisson stream of solve requests of mixed grid
sizes fed in real time to the library's continuous-batching server
(nmg_server_*), reporting throughput and p50/p99 latency.

The scheduling itself (admission into slot pools, one outer iteration per
live request per step, retirement) is in the C library; this module only
generates the stream, submits requests when they are due and collects the
results.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

import nmg_inputs as I

from . import Context, Hierarchy, Server


@dataclass
class Operator:
    """One resident operator class: grid side n, levels, PSF sigma, alpha."""
    n: int
    levels: int
    sigma: float
    alpha: float
    weights: list
    precision: str = "bf16_refine"
    slots: int = 16


@dataclass
class Request:
    t_arrival: float
    op: int
    f: np.ndarray
    u: np.ndarray
    rid: int = -1
    state: int = 0
    info: tuple = ()
    t_submit: float = 0.0
    t_done: float = 0.0


def poisson_stream(ops, n_requests, rate, seed, rhs_batch=8):
    """Arrival times ~ Poisson(rate); operator drawn uniformly (the operator
    list holds the size classes); right-hand sides from the waves generator.
    Right-hand sides are drawn per operator in batches and reused cyclically
    so that generating 10^4 of them stays cheap."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    which = rng.integers(0, len(ops), n_requests)
    pools = {}
    reqs = []
    for i in range(n_requests):
        k = int(which[i])
        o = ops[k]
        if k not in pools:
            f, _ = I.rhs_2d_waves_rects(o.n, rhs_batch, seed * 131 + k, o.sigma)
            pools[k] = f.astype(np.float32)
        f = np.ascontiguousarray(pools[k][i % rhs_batch])
        u = np.zeros((o.n, o.n), dtype=np.float32 if o.precision == "fp32" else np.float64)
        reqs.append(Request(float(t[i]), k, f, u))
    return reqs


def build_server(ctx: Context, ops, budget_bytes, rtol=1e-6, max_cycles=100):
    srv = Server(ctx, budget_bytes, rtol, max_cycles)
    hs, ids = [], []
    for o in ops:
        G = Hierarchy(ctx, dim=2, n=o.n, levels=o.levels, alpha=o.alpha,
                      taps=I.gaussian_taps(o.sigma), precision=o.precision, weights=o.weights)
        hs.append(G)
        ids.append(srv.add_operator(G, o.slots))
    return srv, hs, ids


def run_stream(srv: Server, ids, reqs, time_limit_s=600.0):
    """Submit requests as they come due (wall clock), step the server, collect.
    Returns (elapsed seconds, list of finished Request)."""
    t0 = time.perf_counter()
    nxt = 0
    outstanding = []
    done = []
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        if now > time_limit_s:
            break
        while nxt < len(reqs) and reqs[nxt].t_arrival <= now:
            r = reqs[nxt]
            r.rid = srv.submit(ids[r.op], r.f, r.u)
            outstanding.append(r)
            nxt += 1
        q, running, _ = srv.stats()
        if q + running == 0:
            if nxt < len(reqs):
                time.sleep(max(0.0, min(reqs[nxt].t_arrival - now, 0.01)))
            continue
        if srv.step() > 0:
            keep = []
            for r in outstanding:
                st, info, ts, ta, td = srv.query(r.rid)
                if st == 2:
                    r.state, r.info, r.t_submit, r.t_done = st, info, ts, td
                    done.append(r)
                else:
                    keep.append(r)
            outstanding = keep
    return time.perf_counter() - t0, done


def latency_stats(done):
    lat = np.array([r.t_done - r.t_submit for r in done])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None}
    return {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(lat.mean())}


def size_classes(sizes, weights_for_sigma, alpha=1e-3, precision="bf16_refine", slots=16):
    """Operators for grid sides `sizes`: sigma = max(1, 8 n / 2048) px, 3 levels
    fewer than log2(n) (coarsest grid 8x8)."""
    ops = []
    for n in sizes:
        sigma = max(1.0, 8.0 * n / 2048.0)
        levels = int(math.log2(n)) - 2
        ops.append(Operator(n, levels, sigma, alpha, weights_for_sigma(sigma), precision, slots))
    return ops
