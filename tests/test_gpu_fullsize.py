"""Parity at the full workload sizes, in the launch configuration the bench
times: the whole batch goes through the CUDA path, and sampled right-hand
sides are checked against the FP64 oracle one by one.

* 1D Fredholm problem, n = 256, 3 levels, 16 right-hand sides, fp64: the
  full solve trajectory (cycle counts and iterates) matches the oracle's.
* 2D BTTB 128x128, sigma 2 px, alpha 1e-2, 5 levels, 256 right-hand sides:
  one cycle of the whole batch from zero in fp32 and in the bf16 split
  refinement form (sampled items vs the oracle's cycle), and a full solve
  of the batch whose sampled results meet 1e-6 under the oracle's own apply.
* 2D BTTB 512x512, sigma 4 px, 7 levels, 64 right-hand sides, alpha in
  {1e-1, 1e-2, 1e-3, 1e-4}: one cycle of the whole batch (autotuned launch
  shapes) in the bf16 three-term form, the form with three terms on the
  finest level only and the fp16 pair form against the oracle for four
  sampled items; full solves at every alpha.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import oracle as O  # noqa: E402
from parity_err import rel_both  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402

WDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2603_01064_gb300", "weights")
SAMPLE = [0, 77, 190, 255]


def rel(a, b):
    """Per-RHS max(norm-wise, element-wise) relative error."""
    return rel_both(a, b)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


@pytest.fixture(scope="module")
def c2():
    W = nmg.load_weights(os.path.join(WDIR, "c2_2d_n128_s2_a1e-2.npz"))
    taps = I.gaussian_taps(2.0)
    H = O.build_hierarchy_2d(taps, 128, 1e-2, 5)
    f, _ = I.rhs_2d_ellipses_grf(128, 256, seed=1002, sigma=2.0)
    return W, taps, H, f


def test_1d_full_trajectory_fp64(ctx):
    W = nmg.load_weights(os.path.join(WDIR, "c1_1d_n256_a1e-3.npz"))
    col = I.kernel_column_1d(256)
    H = O.build_hierarchy_1d(col, 1e-3, 3)
    G = nmg.Hierarchy(ctx, dim=1, n=256, levels=3, alpha=1e-3, taps=col, precision="fp64",
                      weights=W)
    f, _ = I.rhs_1d_sines_steps(256, 16, seed=1001)
    fd = torch.tensor(f, dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(fd)
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=60)
    u_o, cyc_o, rr_o = O.solve(H, W, f, rtol=1e-6, max_cycles=60)
    assert np.all(st == 0)
    assert np.array_equal(cyc, cyc_o)
    assert np.max(rel(ud.cpu().numpy(), u_o)) < 1e-10
    assert np.max(np.abs(rr - rr_o) / rr_o) < 1e-6


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("bf16_refine", 1e-3)])
def test_2d_full_batch_one_cycle_sampled(ctx, c2, prec, tol):
    """fp32 bar 1e-4 at this size: trained smoothers amplify fp32 rounding of
    the first cycle from zero to ~2e-5 (their output carries a large part
    the filter removes)."""
    W, taps, H, f = c2
    G = nmg.Hierarchy(ctx, dim=2, n=128, levels=5, alpha=1e-2, taps=taps, precision=prec,
                      weights=W)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    ud = torch.zeros((256, 128, 128), dtype=torch.float32 if prec == "fp32" else torch.float64,
                     device="cuda")
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    u = ud[SAMPLE].double().cpu().numpy()
    ref = O.nmgf(H, W, 0, None, fd[SAMPLE].double().cpu().numpy())
    assert np.max(rel(u, ref)) < tol


@pytest.mark.parametrize("prec", ["fp32", "bf16_refine", "bf16fast_refine"])
def test_2d_full_batch_solve_sampled(ctx, c2, prec):
    W, taps, H, f = c2
    G = nmg.Hierarchy(ctx, dim=2, n=128, levels=5, alpha=1e-2, taps=taps, precision=prec,
                      weights=W)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    ud = torch.zeros((256, 128, 128), dtype=torch.float32 if prec == "fp32" else torch.float64,
                     device="cuda")
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=100)
    assert np.all(st == 0) and np.all(rr <= 1e-6)
    rr_o = O.relres(H, fd[SAMPLE].double().cpu().numpy(), ud[SAMPLE].double().cpu().numpy())
    # fp32 iterates are stored in fp32: their true residual may sit a little
    # above the fp32-computed one
    assert np.all(rr_o <= (1.5e-6 if prec == "fp32" else 1.01e-6)), rr_o


# ---------------------------------------------------------------------------
# 2D BTTB 512x512, sigma 4 px, 7 levels, 64 right-hand sides, alpha sweep
# ---------------------------------------------------------------------------

C3_SAMPLE = [0, 21, 42, 63]


@pytest.fixture(scope="module")
def c3f():
    f, _ = I.rhs_2d_waves_rects(512, 64, seed=1003, sigma=4.0)
    return f


# The bf16 form carries every operand as three bf16 terms (numpy emulation
# of its six products: about 1e-5 after one cycle at every alpha).  The
# pair form bf16x3_refine (2^-16 .. 2^-18 per operand) leaves 1.3e-3 at
# alpha 1e-3 and 1.8e-3 element-wise at alpha 1e-4 (an image corner): the
# trained smoothers amplify operand rounding; it meets the 1e-3 bar at
# alpha 1e-1 and 1e-2 only.
@pytest.mark.parametrize("alpha,prec,tol", [(1e-1, "bf16_refine", 1e-3), (1e-2, "bf16_refine", 1e-3),
                                            (1e-3, "bf16_refine", 1e-3), (1e-4, "bf16_refine", 1e-3),
                                            (1e-1, "bf16x3_refine", 1e-3), (1e-2, "fp32", 1e-4),
                                            (1e-1, "fp16_refine", 1e-3), (1e-2, "fp16_refine", 1e-3),
                                            (1e-3, "fp16_refine", 1e-3), (1e-4, "fp16_refine", 1e-3),
                                            (1e-1, "bf16top_refine", 1e-3), (1e-2, "bf16top_refine", 1e-3),
                                            (1e-3, "bf16top_refine", 1e-3), (1e-4, "bf16top_refine", 1e-3)])
def test_512_full_batch_one_cycle_sampled(ctx, c3f, alpha, prec, tol):
    W = nmg.load_weights(os.path.join(WDIR, f"c3_2d_n512_s4_a{alpha:.0e}".replace("e-0", "e-") + ".npz"))
    taps = I.gaussian_taps(4.0)
    H = O.build_hierarchy_2d(taps, 512, alpha, 7)
    G = nmg.Hierarchy(ctx, dim=2, n=512, levels=7, alpha=alpha, taps=taps, precision=prec,
                      weights=W)
    G.autotune(64)
    fd = torch.tensor(c3f, dtype=torch.float32, device="cuda")
    ud = torch.zeros((64, 512, 512), dtype=torch.float32 if prec == "fp32" else torch.float64,
                     device="cuda")
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    u = ud[C3_SAMPLE].double().cpu().numpy()
    ref = O.nmgf(H, W, 0, None, fd[C3_SAMPLE].double().cpu().numpy())
    assert np.max(rel(u, ref)) < tol


@pytest.mark.parametrize("alpha,max_cycles", [(1e-1, 100), (1e-2, 100), (1e-3, 250), (1e-4, 400)])
def test_512_full_batch_solve_sampled(ctx, c3f, alpha, max_cycles):
    """Every alpha of the sweep reaches 1e-6 on the whole 64-RHS batch
    (checked with the oracle's own apply); about 50 cycles at alpha 1e-3 and
    300 at alpha 1e-4."""
    W = nmg.load_weights(os.path.join(WDIR, f"c3_2d_n512_s4_a{alpha:.0e}".replace("e-0", "e-") + ".npz"))
    taps = I.gaussian_taps(4.0)
    H = O.build_hierarchy_2d(taps, 512, alpha, 7)
    G = nmg.Hierarchy(ctx, dim=2, n=512, levels=7, alpha=alpha, taps=taps,
                      precision="bf16_refine", weights=W)
    fd = torch.tensor(c3f, dtype=torch.float32, device="cuda")
    ud = torch.zeros((64, 512, 512), dtype=torch.float64, device="cuda")
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=max_cycles)
    assert np.all(st == 0) and np.all(rr <= 1e-6)
    rr_o = O.relres(H, fd[C3_SAMPLE].double().cpu().numpy(), ud[C3_SAMPLE].cpu().numpy())
    assert np.all(rr_o <= 1.01e-6), rr_o
    # the compensated outer residual (w = 16 stencil) reports the residual
    # the oracle's fp64 apply finds for the same iterate
    assert np.max(np.abs(rr_o - rr[C3_SAMPLE]) / rr_o) < 1e-3


def test_512_refinement_step_from_nonzero_state(ctx, c3f):
    """One refinement step (compensated residual r = f - A u with the
    half-width-16 stencil, inner cycle on r, fp64 update) from a nonzero u:
    its increment against the oracle cycle's from the same state, at the
    bf16 form's 1e-4."""
    alpha = 1e-2
    W = nmg.load_weights(os.path.join(WDIR, "c3_2d_n512_s4_a1e-2.npz"))
    taps = I.gaussian_taps(4.0)
    H = O.build_hierarchy_2d(taps, 512, alpha, 7)
    G = nmg.Hierarchy(ctx, dim=2, n=512, levels=7, alpha=alpha, taps=taps,
                      precision="bf16_refine", weights=W)
    fd = torch.tensor(c3f[:8], dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(9)
    u0 = 0.3 * rng.standard_normal((8, 512, 512))
    ud = torch.tensor(u0, dtype=torch.float64, device="cuda")
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    k = [0, 5]
    ref = O.nmgf(H, W, 0, u0[k], fd[k].double().cpu().numpy())
    # the step's increments (u0 itself would hide an error in them)
    assert np.max(rel(ud[k].cpu().numpy() - u0[k], ref - u0[k])) < 1e-4
