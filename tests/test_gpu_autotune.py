"""Autotuner: the chosen launch shapes are valid candidates, a cache file
round-trips them, and solves after tuning agree with untuned solves (the
shapes change only the grouping of partial sums)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


def hier(ctx, prec):
    return nmg.Hierarchy(ctx, dim=2, n=128, levels=5, alpha=1e-2, taps=I.gaussian_taps(2.0),
                         precision=prec, weights=I.random_cnn_weights(2, 4, seed=3, scale=0.3))


@pytest.mark.parametrize("prec", ["fp64", "bf16_refine"])
def test_autotune_choices_and_results(ctx, prec, tmp_path):
    f, _ = I.rhs_2d_ellipses_grf(128, 4, seed=8, sigma=2.0)
    dt = torch.float64 if prec == "fp64" else torch.float32
    fd = torch.tensor(f, dtype=dt, device="cuda")
    u0 = torch.zeros((4, 128, 128), dtype=torch.float64, device="cuda")
    G = hier(ctx, prec)
    u_ref = u0.clone()
    for _ in range(3):
        G.cycle(fd, u_ref)
    cache = str(tmp_path / "tune.txt")
    G.autotune(4, cache)
    for l in range(5):
        t = G.tuning(l)
        assert t["res_tile"] in (16, 32, 64)
        if l < 4:
            assert t["rst_tile"] in (8, 16, 32) and t["filt_mode"] in (0, 1, 2)
    u = u0.clone()
    for _ in range(3):
        G.cycle(fd, u)
    torch.cuda.synchronize()
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert (torch.norm(u - u_ref) / torch.norm(u_ref)).item() < tol
    # a second hierarchy of the same shape reads the cached choices
    G2 = hier(ctx, prec)
    G2.autotune(4, cache)
    for l in range(5):
        assert G2.tuning(l) == G.tuning(l)
    assert len(open(cache).read().strip().splitlines()) == 1
