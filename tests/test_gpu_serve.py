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
