"""GPU parity of the classical comparators (nmg_solve_mg_jacobi: the V-cycle
of Algorithm 1 with weighted Jacobi smoothing; nmg_solve_cg: conjugate
gradients) against the oracle's textbook versions (oracle/classical.py), on
the same hierarchies, through the C ABI.

Tolerances as for the neural cycle: fp64 one cycle / iterates 1e-10, fp32
1e-5 (max of norm-wise and element-wise relative error); fp64 solves take
the oracle's cycle / iteration counts; converged solves meet 1e-6 under the
oracle's own apply.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import oracle as O  # noqa: E402
from parity_err import rel_both  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402

TOL = {"fp64": 1e-10, "fp32": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


def make(ctx, prec, dim, n, levels, sigma, alpha):
    if dim == 2:
        taps = I.gaussian_taps(sigma)
        H = O.build_hierarchy_2d(taps, n, alpha, levels)
        W = I.random_cnn_weights(2, levels - 1, seed=2)
    else:
        taps = I.kernel_column_1d(n)
        H = O.build_hierarchy_1d(taps, alpha, levels)
        W = I.random_cnn_weights(1, levels - 1, seed=2)
    G = nmg.Hierarchy(ctx, dim=dim, n=n, levels=levels, alpha=alpha, taps=taps, precision=prec,
                      weights=W)
    return H, G


def rhs(dim, n, B, seed, sigma):
    if dim == 2:
        return I.rhs_2d_ellipses_grf(n, B, seed=seed, sigma=sigma)[0]
    return I.rhs_1d_sines_steps(n, B, seed=seed)[0]


CASES = [(2, 64, 4, 1.0, 1e-1), (1, 256, 3, 0.0, 1e-1), (2, 256, 4, 4.0, 1e-2)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nu", [(5, 0), (2, 1)])
def test_vcycle_one_cycle(ctx, prec, case, nu):
    """One V-cycle from a random state (the last case: PSF half-width 16,
    whose fine-level residual takes the wide strip kernel)."""
    dim, n, L, sigma, alpha = case
    H, G = make(ctx, prec, dim, n, L, sigma, alpha)
    rng = np.random.default_rng(n + L)
    shape = (3, n, n) if dim == 2 else (3, n)
    f = rhs(dim, n, 3, 31, sigma)
    u0 = 0.3 * rng.standard_normal(shape)
    fd = torch.tensor(f, dtype=DT[prec], device="cuda")
    ud = torch.tensor(u0, dtype=DT[prec], device="cuda")
    f_in, u_in = fd.double().cpu().numpy(), ud.double().cpu().numpy()
    cyc, st, rr = G.solve_mg_jacobi(fd, ud, rtol=0.0, max_cycles=1, nu1=nu[0], nu2=nu[1])
    assert np.all(cyc == 1)
    ref = O.mg_cycle(H, 0, u_in, f_in, nu[0], nu[1])
    assert np.max(rel_both(ud.double().cpu().numpy(), ref)) < TOL[prec]


def test_vcycle_solve_takes_the_oracle_cycles(ctx):
    H, G = make(ctx, "fp64", 2, 64, 4, 1.0, 1e-1)
    f = rhs(2, 64, 4, 32, 1.0)
    fd = torch.tensor(f, dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(fd)
    cyc, st, rr = G.solve_mg_jacobi(fd, ud, rtol=1e-6, max_cycles=500)
    u_o, cyc_o, rr_o = O.mg_solve(H, f, rtol=1e-6, max_cycles=500)
    assert np.all(st == nmg.CONVERGED) and np.array_equal(cyc, cyc_o)
    assert np.all(O.relres(H, f, ud.cpu().numpy()) <= 1.001e-6)
    assert np.max(rel_both(ud.cpu().numpy(), u_o)) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_cg_iterates(ctx, prec, case):
    """Five CG iterations from zero against the oracle's."""
    dim, n, L, sigma, alpha = case
    H, G = make(ctx, prec, dim, n, L, sigma, alpha)
    f = rhs(dim, n, 3, 33, sigma)
    fd = torch.tensor(f, dtype=DT[prec], device="cuda")
    ud = torch.zeros_like(fd)
    its, st, rr = G.solve_cg(fd, ud, rtol=0.0, max_iters=5)
    assert np.all(its == 5)
    u_o, its_o, rr_o = O.cg(H, fd.double().cpu().numpy(), rtol=0.0, max_iters=5)
    assert np.max(rel_both(ud.double().cpu().numpy(), u_o)) < 10 * TOL[prec]
    assert np.max(np.abs(rr - rr_o) / rr_o) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cg_solve(ctx, prec):
    H, G = make(ctx, prec, 2, 128, 5, 2.0, 1e-2)
    f = rhs(2, 128, 4, 34, 2.0)
    fd = torch.tensor(f, dtype=DT[prec], device="cuda")
    ud = torch.zeros_like(fd)
    its, st, rr = G.solve_cg(fd, ud, rtol=1e-6, max_iters=2000)
    assert np.all(st == nmg.CONVERGED) and np.all(rr <= 1e-6)
    rr_true = O.relres(H, fd.double().cpu().numpy(), ud.double().cpu().numpy())
    # fp32: the recurred residual drifts from the true one by a few fp32
    # roundings of A u relative to f
    assert np.all(rr_true <= (1.001e-6 if prec == "fp64" else 1e-5)), rr_true
    if prec == "fp64":
        _, its_o, _ = O.cg(H, f, rtol=1e-6, max_iters=2000)
        assert np.array_equal(its, its_o)
