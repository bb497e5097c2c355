"""FNO smoother (Section 3.1, Appendix A) through the C ABI against the FP64
oracle, on seeded random FNO weights (width 8, 2 Fourier layers, 4 modes,
3x3 W term) and a 2D BTTB operator (64x64, sigma 2 px, alpha 1e-2, 3 levels):

* the smoother alone on each smoother level: fp64 1e-12, fp32 2e-5;
* one whole cycle from zero: fp64 1e-10, fp32 1e-5 (the bars of the CNN
  path's parity tests);
* a ragged batch with an all-zero right-hand side (h = 0 there);
* setup rejects modes beyond the coarsest smoother level, the 16-bit forms
  and a weight count that does not match;
* the trained FNO smoothers of the 128x128 operator (sigma 2 px, alpha
  1e-2, 5 levels): one fp32 cycle against the oracle, and a solve to 1e-6.
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

N, L, ALPHA, SIGMA = 64, 3, 1e-2, 2.0
DT = {"fp64": torch.float64, "fp32": torch.float32}
TOL_SMOOTH = {"fp64": 1e-12, "fp32": 2e-5}
TOL_CYCLE = {"fp64": 1e-10, "fp32": 1e-5}


def rel(a, b):
    """Per-RHS max(norm-wise, element-wise) relative error."""
    return rel_both(a, b)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


@pytest.fixture(scope="module")
def setup():
    taps = I.gaussian_taps(SIGMA)
    W = I.random_fno_weights(L - 1, seed=31, width=8, layers=2, modes=4, ksize=3)
    H = O.build_hierarchy_2d(taps, N, ALPHA, L)
    f, _ = I.rhs_2d_ellipses_grf(N, 5, seed=1021, sigma=SIGMA)
    return taps, W, H, f


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fno_smoother_matches_oracle(ctx, setup, prec):
    taps, W, H, f = setup
    G = nmg.Hierarchy(ctx, dim=2, n=N, levels=L, alpha=ALPHA, taps=taps, precision=prec,
                      weights=W)
    rng = np.random.default_rng(7)
    for lvl in range(L - 1):
        m = N >> lvl
        b = rng.standard_normal((3, m, m))
        b[1] = 0.0  # ||b|| = 0 gives h = 0
        bd = torch.tensor(b, dtype=DT[prec], device="cuda")
        hd = torch.full_like(bd, 7.0)
        G.smooth(lvl, bd, hd)
        torch.cuda.synchronize()
        h = hd.double().cpu().numpy()
        ref = O.smoother(W[lvl], b)
        assert np.all(h[1] == 0.0)
        keep = [0, 2]
        assert np.max(rel(h[keep], ref[keep])) < TOL_SMOOTH[prec], lvl


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fno_one_cycle_matches_oracle(ctx, setup, prec):
    taps, W, H, f = setup
    G = nmg.Hierarchy(ctx, dim=2, n=N, levels=L, alpha=ALPHA, taps=taps, precision=prec,
                      weights=W)
    fd = torch.tensor(f, dtype=DT[prec], device="cuda")
    ud = torch.zeros_like(fd)
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    ref = O.nmgf(H, W, 0, None, f)
    assert np.max(rel(ud.double().cpu().numpy(), ref)) < TOL_CYCLE[prec]


def test_fno_setup_rejects(ctx, setup):
    taps, W, H, f = setup
    big = I.random_fno_weights(L - 1, seed=1, width=4, layers=1, modes=17, ksize=3)
    with pytest.raises(nmg.NMGError):  # 2 x 17 > 32, the side of the coarsest smoother level
        nmg.Hierarchy(ctx, dim=2, n=N, levels=L, alpha=ALPHA, taps=taps, precision="fp32",
                      weights=big)
    with pytest.raises(nmg.NMGError):  # the FNO smoother runs in fp64 / fp32 only
        nmg.Hierarchy(ctx, dim=2, n=N, levels=L, alpha=ALPHA, taps=taps,
                      precision="bf16_refine", weights=W)
    with pytest.raises(nmg.NMGError):  # one smoother level too few
        nmg.Hierarchy(ctx, dim=2, n=N, levels=L + 1, alpha=ALPHA, taps=taps, precision="fp32",
                      weights=W)


# ---------------------------------------------------------------------------
# trained FNO smoothers (128x128, sigma 2 px, alpha 1e-2, 5 levels)
# ---------------------------------------------------------------------------

FNO_W = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                     "paper_2603_01064_gb300", "weights", "c2f_2d_n128_s2_a1e-2_fno.npz")


def test_fno_trained_cycle_and_solve(ctx):
    """The trained FNO smoothers: one fp32 cycle of 2 sampled right-hand sides
    against the oracle's cycle (1e-4: trained smoothers amplify fp32
    rounding), and the whole 32-RHS batch solved to 1e-6 with the oracle's
    own apply confirming the residual."""
    W = nmg.load_weights(FNO_W)
    taps = I.gaussian_taps(2.0)
    H = O.build_hierarchy_2d(taps, 128, 1e-2, 5)
    f, _ = I.rhs_2d_ellipses_grf(128, 32, seed=1002, sigma=2.0)
    G = nmg.Hierarchy(ctx, dim=2, n=128, levels=5, alpha=1e-2, taps=taps, precision="fp32",
                      weights=W)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    ud = torch.zeros_like(fd)
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    ref = O.nmgf(H, W, 0, None, f[:2])
    assert np.max(rel(ud[:2].double().cpu().numpy(), ref)) < 1e-4
    ud.zero_()
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=100)
    assert np.all(st == 0) and np.all(rr <= 1e-6)
    assert np.all(O.relres(H, f[[0, 31]], ud[[0, 31]].double().cpu().numpy()) <= 1.5e-6)
