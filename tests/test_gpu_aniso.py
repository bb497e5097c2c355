"""The anisotropic regularisation of Section 4.1 (A = alpha D + hK, D the
tridiagonal flux form of -(a u')' with a(z) = 1 + 0.5 sin(2 pi z)) through
the C ABI, against the FP64 oracle:

* fp64, n = 256, 3 levels, alpha 1e-5, 16 right-hand sides, trained 1D CNN
  smoothers: the whole solve trajectory (cycle counts, iterates, residuals);
* fp32: one cycle from zero, sampled against the oracle's cycle;
* setup rejects a tridiagonal D of the wrong length and D in 2D.
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

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2603_01064_gb300", "weights", "c1a_1d_n256_aniso_a1e-5.npz")
N, L, ALPHA = 256, 3, 1e-5


def rel(a, b):
    """Per-RHS max(norm-wise, element-wise) relative error."""
    return rel_both(a, b)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


@pytest.fixture(scope="module")
def prob():
    col = I.kernel_column_1d(N)
    reg = I.aniso_regularisation_1d(N)
    W = nmg.load_weights(WEIGHTS)
    H = O.build_hierarchy_1d(col, ALPHA, L, reg=reg)
    f, _ = I.rhs_1d_sines_steps(N, 16, seed=1011)
    return col, reg, W, H, f


def test_aniso_full_trajectory_fp64(ctx, prob):
    col, reg, W, H, f = prob
    G = nmg.Hierarchy(ctx, dim=1, n=N, levels=L, alpha=ALPHA, taps=col, precision="fp64",
                      weights=W, reg=reg)
    fd = torch.tensor(f, dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(fd)
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=60)
    u_o, cyc_o, rr_o = O.solve(H, W, f, rtol=1e-6, max_cycles=60)
    assert np.all(st == 0)
    assert np.array_equal(cyc, cyc_o)
    assert np.max(rel(ud.cpu().numpy(), u_o)) < 1e-10
    assert np.max(np.abs(rr - rr_o) / rr_o) < 1e-6
    # the operator the library built is the oracle's level by level
    for l in range(L):
        assert np.abs(G.level_dense(l) - H.ops[l]).max() <= 1e-13 * np.abs(H.ops[l]).max()


def test_aniso_one_cycle_fp32(ctx, prob):
    col, reg, W, H, f = prob
    G = nmg.Hierarchy(ctx, dim=1, n=N, levels=L, alpha=ALPHA, taps=col, precision="fp32",
                      weights=W, reg=reg)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    ud = torch.zeros_like(fd)
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    ref = O.nmgf(H, W, 0, None, fd.double().cpu().numpy())
    assert np.max(rel(ud.double().cpu().numpy(), ref)) < 1e-4


def test_aniso_setup_rejects_bad_reg(ctx, prob):
    col, reg, W, H, f = prob
    with pytest.raises(nmg.NMGError):
        nmg.Hierarchy(ctx, dim=1, n=N, levels=L, alpha=ALPHA, taps=col, precision="fp64",
                      weights=W, reg=(reg[0][:-1], reg[1]))
    taps = I.gaussian_taps(2.0)
    W2 = I.random_cnn_weights(2, 1, seed=3)
    with pytest.raises(nmg.NMGError):
        nmg.Hierarchy(ctx, dim=2, n=64, levels=2, alpha=1e-2, taps=taps, precision="fp32",
                      weights=W2, reg=reg)
