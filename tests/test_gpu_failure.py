"""Failure handling of the solve on the GPU, made on the host or with a
wait that nothing ends, never with a device fault (per right-hand-side
outcomes of Section 3.2's outer iteration, and the bounded device waits of
the tensor-core smoother):

* a right-hand side containing a NaN is reported NMG_DIVERGED with a NaN
  relative residual before any cycle runs; the other right-hand sides of
  the same batch converge, bitwise as when each is solved alone;
* a max_cycles cut-off reports NMG_NOT_CONVERGED after exactly max_cycles
  cycles, with the relative residual of the last iterate above the
  tolerance;
* a tensor-core wait that runs out (the stall hook: the MMA issuers wait on
  a barrier that nothing arrives at, bounded by a 20 ms wait limit) makes
  the solve return NMG_ERR_TIMEOUT; the launches drained their copies and
  released their tensor memory, so the same context and hierarchy then
  solve normally, bitwise as a fresh context does.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import oracle as O  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402

WDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2603_01064_gb300", "weights")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


@pytest.fixture(scope="module")
def c2():
    W = nmg.load_weights(os.path.join(WDIR, "c2_2d_n128_s2_a1e-2.npz"))
    f, _ = I.rhs_2d_ellipses_grf(128, 3, seed=606, sigma=2.0)
    return W, f


def hier(ctx, W, prec):
    return nmg.Hierarchy(ctx, dim=2, n=128, levels=5, alpha=1e-2, taps=I.gaussian_taps(2.0),
                         precision=prec, weights=W)


def udtype(prec):
    return torch.float32 if prec == "fp32" else torch.float64


@pytest.mark.parametrize("prec", ["fp32", "bf16_refine"])
def test_nan_rhs_diverged_others_unaffected(ctx, c2, prec):
    W, f = c2
    G = hier(ctx, W, prec)
    fb = f.copy()
    fb[1, 40, 77] = np.nan
    fd = torch.tensor(fb, dtype=torch.float32, device="cuda")
    ud = torch.zeros((3, 128, 128), dtype=udtype(prec), device="cuda")
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=100)
    assert st[1] == nmg.DIVERGED and np.isnan(rr[1]) and cyc[1] == 0
    assert st[0] == nmg.CONVERGED and st[2] == nmg.CONVERGED
    assert rr[0] <= 1e-6 and rr[2] <= 1e-6
    for i in (0, 2):
        ui = torch.zeros((1, 128, 128), dtype=udtype(prec), device="cuda")
        ci, si, ri = G.solve(fd[i:i + 1].clone(), ui, rtol=1e-6, max_cycles=100)
        assert si[0] == nmg.CONVERGED and ci[0] == cyc[i] and ri[0] == rr[i]
        assert torch.equal(ui[0], ud[i])
    G.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16_refine"])
def test_max_cycles_not_converged(ctx, c2, prec):
    W, f = c2
    G = hier(ctx, W, prec)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    ud = torch.zeros((3, 128, 128), dtype=udtype(prec), device="cuda")
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=3)
    assert np.all(st == nmg.NOT_CONVERGED) and np.all(cyc == 3) and np.all(rr > 1e-6)
    # the reported residual is the last iterate's (checked with the oracle's apply)
    H = O.build_hierarchy_2d(I.gaussian_taps(2.0), 128, 1e-2, 5)
    rr_o = O.relres(H, fd.double().cpu().numpy(), ud.double().cpu().numpy())
    assert np.max(np.abs(rr_o - rr) / rr_o) < (1e-4 if prec == "fp32" else 1e-6)
    G.close()


def test_wait_timeout_then_recovers(c2):
    W, f = c2
    c = nmg.Context(0)
    G = hier(c, W, "bf16_refine")
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    ud = torch.zeros((3, 128, 128), dtype=torch.float64, device="cuda")
    c.set_wait_limit(20_000_000)
    c.inject_stall(True)
    try:
        with pytest.raises(nmg.NMGError) as e:
            G.solve(fd, ud, rtol=1e-6, max_cycles=100)
        assert e.value.code == -5  # NMG_ERR_TIMEOUT
    finally:
        c.inject_stall(False)
        c.set_wait_limit(2_000_000_000)
    ud.zero_()
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=100)
    assert np.all(st == nmg.CONVERGED)
    c2x = nmg.Context(0)
    G2 = hier(c2x, W, "bf16_refine")
    u2 = torch.zeros_like(ud)
    cyc2, st2, rr2 = G2.solve(fd, u2, rtol=1e-6, max_cycles=100)
    assert np.array_equal(cyc, cyc2) and torch.equal(ud, u2)
    with pytest.raises(nmg.NMGError):
        c.set_wait_limit(0)
    G2.close()
    G.close()
