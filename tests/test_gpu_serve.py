"""Serving loop with continuous batching: requests of two grid sizes arrive
while others are running, are admitted into slots as they free up, and each
result equals the result of solving that right-hand side alone (the slots
are computed independently; tolerance 1e-12 relative, expected bitwise)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402
from paper_2603_01064_gb300 import serve  # noqa: E402

WDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2603_01064_gb300", "weights")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


@pytest.mark.parametrize("prec", ["bf16_refine", "fp32"])
def test_stream_results_equal_solo(ctx, prec):
    W = nmg.load_weights(os.path.join(WDIR, "c2_2d_n128_s2_a1e-2.npz"))
    ops = [serve.Operator(64, 4, 2.0, 1e-2, W, prec, slots=3),
           serve.Operator(128, 5, 2.0, 1e-2, W, prec, slots=2)]
    srv, hs, ids = serve.build_server(ctx, ops, budget_bytes=8 << 30)
    reqs = serve.poisson_stream(ops, 24, rate=2000.0, seed=9, rhs_batch=5)
    elapsed, done = serve.run_stream(srv, ids, reqs, time_limit_s=120)
    assert len(done) == len(reqs)
    q, running, used = srv.stats()
    assert q == 0 and running == 0 and 0 < used <= 8 << 30
    # solve every right-hand side alone on its own hierarchy
    for r in reqs:
        G = hs[r.op]
        fd = torch.tensor(r.f[None], device="cuda")
        ud = torch.zeros((1,) + r.f.shape, dtype=torch.float32 if prec == "fp32" else torch.float64,
                         device="cuda")
        cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=100)
        assert st[0] == 0 and r.info[1] == 0
        assert r.info[0] == cyc[0]
        u_alone = ud[0].cpu().numpy()
        assert np.linalg.norm(r.u - u_alone) <= 1e-12 * np.linalg.norm(u_alone)
    srv.close()


def test_budget_bounds_admission(ctx):
    W = nmg.load_weights(os.path.join(WDIR, "c2_2d_n128_s2_a1e-2.npz"))
    srv = nmg.Server(ctx, budget_bytes=1 << 20)
    G = nmg.Hierarchy(ctx, dim=2, n=128, levels=5, alpha=1e-2, taps=I.gaussian_taps(2.0),
                      precision="bf16_refine", weights=W)
    with pytest.raises(nmg.NMGError) as e:
        srv.add_operator(G, 4)
    assert e.value.code == -2
    srv.close()


def test_pools_grow_as_requests_wait(ctx):
    """An operator allowed 16 slots starts with 4; a burst of 20 requests makes
    the pool grow at the next steps (free device memory permitting, which it
    does here), every request is served, and each result equals solving that
    right-hand side alone."""
    W = nmg.load_weights(os.path.join(WDIR, "c2_2d_n128_s2_a1e-2.npz"))
    ops = [serve.Operator(128, 5, 2.0, 1e-2, W, "bf16_refine", slots=16)]
    srv, hs, ids = serve.build_server(ctx, ops, budget_bytes=0)
    _, _, used0 = srv.stats()
    reqs = serve.poisson_stream(ops, 20, rate=1e6, seed=19, rhs_batch=6)
    elapsed, done = serve.run_stream(srv, ids, reqs, time_limit_s=120)
    assert len(done) == len(reqs)
    _, _, used1 = srv.stats()
    assert used1 > used0  # the pool grew beyond its first 4 slots
    G = hs[0]
    for r in reqs:
        fd = torch.tensor(r.f[None], device="cuda")
        ud = torch.zeros((1,) + r.f.shape, dtype=torch.float64, device="cuda")
        cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=100)
        assert r.info[1] == st[0] == 0 and r.info[0] == cyc[0]
        assert np.array_equal(r.u, ud[0].cpu().numpy())
    srv.close()


def test_2048_request_in_the_mix(ctx):
    """A 2048 x 2048 operator (9 levels, PSF sigma 8 px, alpha 1e-3; seeded
    untrained smoothers, so the server's cycle limit of 2 ends the requests)
    served together with a 64 x 64 one: every result equals solving that
    right-hand side alone with the same cycle limit."""
    W9 = I.random_cnn_weights(2, 8, seed=41)
    W4 = I.random_cnn_weights(2, 3, seed=42)
    ops = [serve.Operator(2048, 9, 8.0, 1e-3, W9, "bf16_refine", slots=2),
           serve.Operator(64, 4, 1.0, 1e-3, W4, "bf16_refine", slots=4)]
    srv, hs, ids = serve.build_server(ctx, ops, budget_bytes=0, max_cycles=2)
    reqs = serve.poisson_stream(ops, 6, rate=1e6, seed=23, rhs_batch=3)
    assert {r.op for r in reqs} == {0, 1}
    elapsed, done = serve.run_stream(srv, ids, reqs, time_limit_s=300)
    assert len(done) == len(reqs)
    for r in reqs:
        G = hs[r.op]
        fd = torch.tensor(r.f[None], device="cuda")
        ud = torch.zeros((1,) + r.f.shape, dtype=torch.float64, device="cuda")
        cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=2)
        assert r.info[0] == cyc[0] == 2 and r.info[1] == st[0]
        assert np.array_equal(r.u, ud[0].cpu().numpy())
    srv.close()
