"""Pins of the oracle's classical comparators (oracle/classical.py): the
weighted Jacobi smoother of Section 2.2, the multigrid V-cycle of Algorithm 1
and conjugate gradients, each against what the paper or the mathematics fixes
independently of the oracle's own code: the paper's printed Jacobi symbol
values, the textbook error-propagation product of the V-cycle built from
brute-force dense matrices, the neural cycle's own code path with a linear
Jacobi 'network', Gershgorin's bound, the Krylov-subspace optimality and
finite termination of CG, and LU solutions."""
import json
import os

import numpy as np
import pytest

import nmg_inputs as I
import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dense_2d(H, l):
    """A_l = alpha M (x) M + K (x) K as an explicit dense matrix (row-major
    grid order)."""
    M, K = H.ops[l]
    return H.alpha * np.kron(M, M) + np.kron(K, K)


def test_jacobi_symbol_golden():
    """Section 2.2: one weighted Jacobi step (omega = 1/2) of the oracle on the
    periodic model matrix tridiag(-1, 2 + alpha, -1), applied to the error
    modes (-1)^k and 1 (y = 0), multiplies them by the printed extreme symbol
    values 1 - (4 + alpha) / (4 + 2 alpha) and 1 - alpha / (4 + 2 alpha)."""
    with open(os.path.join(GOLDEN, "jacobi_symbol.json")) as fh:
        g = json.load(fh)
    n = 16
    for case in g["cases"]:
        alpha = case["alpha"]
        A = (2 + alpha) * np.eye(n) - np.roll(np.eye(n), 1, 1) - np.roll(np.eye(n), -1, 1)
        d = np.full(n, 2 + alpha)
        for mode, printed in [((-1.0) ** np.arange(n), case["mu_min"]), (np.ones(n), case["mu_max"])]:
            x1 = O.jacobi_sweeps(lambda v: v @ A.T, d, mode[None], np.zeros((1, n)), 1, 0.5)
            assert np.allclose(x1[0], printed * mode, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_level_diagonal_and_weight_from_dense(dim):
    if dim == 2:
        H = O.build_hierarchy_2d(I.gaussian_taps(1.5), 16, 1e-2, 3)
        dense = [dense_2d(H, l) for l in range(2)]
    else:
        H = O.build_hierarchy_1d(I.kernel_column_1d(64), 1e-3, 3)
        dense = [H.ops[l] for l in range(2)]
    for l, A in enumerate(dense):
        d = O.level_diagonal(H, l).reshape(-1)
        assert np.array_equal(d, np.diag(A))
        rho = np.max(np.sum(np.abs(A), axis=1) / np.diag(A))
        w = O.jacobi_weight(H, l)
        assert abs(w * rho - 1.0) < 1e-13
        # Gershgorin: the weighted Jacobi iteration contracts (omega lambda <= 1)
        lam = np.max(np.linalg.eigvals(np.diag(1 / np.diag(A)) @ A).real)
        assert w * lam <= 1.0 + 1e-12


def test_vcycle_is_textbook_error_propagation():
    """Algorithm 1 with nu1 = 2 pre- and nu2 = 1 post-smoothing steps on a
    three-level 2D hierarchy: x1 - x = E (x0 - x) with E_l = S_l^nu2
    (I - P_l (I - E_{l+1}) A_{l+1}^{-1} R_l A_l) S_l^nu1, S_l = I - omega_l
    D_l^{-1} A_l, E_L = 0, every matrix dense (Kronecker transfers, RAP)."""
    n, L, nu1, nu2 = 16, 3, 2, 1
    H = O.build_hierarchy_2d(I.gaussian_taps(1.0), n, 1e-1, L)
    A = [dense_2d(H, 0)]
    Ps = []
    for l in range(L - 1):
        P = np.kron(O.prolongation((n >> l) // 2), O.prolongation((n >> l) // 2))
        Ps.append(P)
        A.append((P.T / 4) @ A[-1] @ P)

    def E(l):
        if l == L - 1:
            return np.zeros_like(A[l])
        N = A[l].shape[0]
        S = np.eye(N) - O.jacobi_weight(H, l) * np.diag(1 / np.diag(A[l])) @ A[l]
        Ec = E(l + 1)
        C = np.eye(N) - Ps[l] @ (np.eye(Ec.shape[0]) - Ec) @ np.linalg.solve(A[l + 1], (Ps[l].T / 4) @ A[l])
        return np.linalg.matrix_power(S, nu2) @ C @ np.linalg.matrix_power(S, nu1)

    rng = np.random.default_rng(3)
    xt = rng.standard_normal((2, n * n))
    y = xt @ A[0].T
    x0 = rng.standard_normal((2, n * n))
    x1 = O.mg_cycle(H, 0, x0.reshape(2, n, n), y.reshape(2, n, n), nu1, nu2).reshape(2, -1)
    ref = xt + (x0 - xt) @ E(0).T
    assert np.max(np.abs(x1 - ref)) < 1e-11 * np.max(np.abs(ref))


def test_vcycle_equals_neural_cycle_with_linear_jacobi_network():
    """nu1 = 1, nu2 = 0 on a two-level 1D hierarchy whose fine level has a
    constant diagonal d: Algorithm 1 equals the neural cycle (a different code
    path of the oracle) with the one-layer linear network omega / d and the
    output filter off."""
    n = 64
    H = O.build_hierarchy_1d(I.kernel_column_1d(n, 0.05), 1e-2, 2)
    d = H.ops[0][0, 0]
    w = O.jacobi_weight(H, 0)
    W = [[(np.array([[[0.0, w / d, 0.0]]]), np.array([0.0]))]]
    rng = np.random.default_rng(4)
    y = rng.standard_normal((3, n))
    x0 = rng.standard_normal((3, n))
    a = O.mg_cycle(H, 0, x0, y, 1, 0)
    b = O.nmgf(H, W, 0, x0, y, filt=False)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_mg_solve_reaches_lu_solution():
    n, L, alpha = 32, 3, 1e-1
    H = O.build_hierarchy_2d(I.gaussian_taps(1.0), n, alpha, L)
    f, _ = I.rhs_2d_ellipses_grf(n, 2, seed=7, sigma=1.0)
    u, cyc, rr = O.mg_solve(H, f, rtol=1e-6, max_cycles=500)
    assert np.all(rr <= 1e-6) and np.all(cyc > 1)
    A = dense_2d(H, 0)
    ulu = np.linalg.solve(A, f.reshape(2, -1).T).T
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(u.reshape(2, -1) - ulu, axis=1) / np.linalg.norm(ulu, axis=1)
    assert np.all(err <= kappa * 1e-6)


def test_cg_krylov_optimality():
    """After k steps from zero, CG's iterate minimises the A-norm of the error
    over the Krylov space span{f, A f, ..., A^{k-1} f}: checked against the
    Galerkin solution on an orthonormal basis of that space."""
    n = 48
    H = O.build_hierarchy_1d(I.kernel_column_1d(n), 1e-2, 1)
    A = H.ops[0]
    f = np.random.default_rng(5).standard_normal((1, n))
    for k in range(1, 7):
        u, its, _ = O.cg(H, f, rtol=0.0, max_iters=k)
        assert its[0] == k
        V = np.empty((n, k))
        v = f[0].copy()
        for j in range(k):
            V[:, j] = v
            v = A @ v
        Q, _ = np.linalg.qr(V)
        ref = Q @ np.linalg.solve(Q.T @ A @ Q, Q.T @ f[0])
        assert np.max(np.abs(u[0] - ref)) < 1e-9 * np.max(np.abs(ref))


def test_cg_finite_termination_and_lu():
    """An SPD system of order N is solved in at most N steps (up to rounding);
    the 2D solve to 1e-6 agrees with LU within kappa * 1e-6."""
    n = 12
    H = O.build_hierarchy_1d(I.kernel_column_1d(n, 0.2), 1e-1, 1)
    f = np.random.default_rng(6).standard_normal((2, n))
    u, its, rr = O.cg(H, f, rtol=1e-12, max_iters=3 * n)
    assert np.all(its <= n + 2) and np.all(rr <= 1e-12)
    H2 = O.build_hierarchy_2d(I.gaussian_taps(1.0), 32, 1e-2, 3)
    f2, _ = I.rhs_2d_ellipses_grf(32, 2, seed=8, sigma=1.0)
    u2, its2, rr2 = O.cg(H2, f2, rtol=1e-6, max_iters=1000)
    assert np.all(rr2 <= 1e-6)
    A = dense_2d(H2, 0)
    ulu = np.linalg.solve(A, f2.reshape(2, -1).T).T
    err = np.linalg.norm(u2.reshape(2, -1) - ulu, axis=1) / np.linalg.norm(ulu, axis=1)
    assert np.all(err <= np.linalg.cond(A) * 1e-6)
    # the recurred residual is the true one up to rounding
    assert np.allclose(O.relres(H2, f2, u2), rr2, rtol=1e-6, atol=1e-12)


# ---------------------------------------------------------------------------
# planted mistakes: each makes the named pins above fail (on the CPU)
# ---------------------------------------------------------------------------

from oracle import classical as OC  # noqa: E402

_sweeps = OC.jacobi_sweeps
_weight = OC.jacobi_weight
_apply = OC.apply_level


def sweeps_without_diagonal(apply, d, x, y, nu, omega):
    return _sweeps(apply, np.ones_like(d), x, y, nu, omega)  # x += omega (y - A x)


def weight_from_diagonal_only(H, l):
    return 1.0 / np.max(O.level_diagonal(H, l))


def cycle_restricting_residual_of_guess(H, l, xstar, y, nu1=5, nu2=0, omega=None):
    if l == H.levels - 1:
        B = y.shape[0]
        return O.cholesky_solve(H.chol, y.reshape(B, -1).T).T.reshape(y.shape)
    x0 = np.zeros_like(y) if xstar is None else np.array(xstar, np.float64)
    x = OC.jacobi_smooth(H, l, x0, y, nu1, omega)
    yc = O.restrict(H, l, y - _apply(H, l, x0))  # residual of x* instead of x
    x = x + O.prolong(H, l, cycle_restricting_residual_of_guess(H, l + 1, None, yc, nu1, nu2, omega))
    return OC.jacobi_smooth(H, l, x, y, nu2, omega)


def cg_inverted_beta(H, f, rtol=1e-6, max_iters=10000, u0=None):
    f = np.asarray(f, np.float64)
    u = np.zeros_like(f)
    r = f - _apply(H, 0, u)
    p = r.copy()
    fn = np.linalg.norm(f.reshape(f.shape[0], -1), axis=1)
    its = np.zeros(f.shape[0], dtype=np.int64)
    for b in range(f.shape[0]):
        rr = np.dot(r[b].ravel(), r[b].ravel())
        while np.sqrt(rr) / fn[b] > rtol and its[b] < max_iters:
            Ap = _apply(H, 0, p[b:b + 1])[0]
            a = rr / np.dot(p[b].ravel(), Ap.ravel())
            u[b] += a * p[b]
            r[b] -= a * Ap
            rr_new = np.dot(r[b].ravel(), r[b].ravel())
            p[b] = r[b] + (rr / rr_new) * p[b]  # beta inverted
            rr = rr_new
            its[b] += 1
    return u, its, np.linalg.norm(r.reshape(f.shape[0], -1), axis=1) / fn


CLASSICAL_MUTANTS = {
    "Jacobi without the diagonal": ("jacobi_sweeps", sweeps_without_diagonal,
                                    [test_jacobi_symbol_golden,
                                     test_vcycle_is_textbook_error_propagation]),
    "Jacobi weight from the diagonal alone": ("jacobi_weight", weight_from_diagonal_only,
                                              [lambda: test_level_diagonal_and_weight_from_dense(2)]),
    "V-cycle restricts the residual of the guess": ("mg_cycle", cycle_restricting_residual_of_guess,
                                                    [test_vcycle_is_textbook_error_propagation]),
    "CG with the inverse beta": ("cg", cg_inverted_beta, [test_cg_krylov_optimality]),
}


@pytest.mark.parametrize("mutant", sorted(CLASSICAL_MUTANTS))
def test_classical_pins_catch_planted_mistake(monkeypatch, mutant):
    name, fn, pins = CLASSICAL_MUTANTS[mutant]
    monkeypatch.setattr(OC, name, fn)
    monkeypatch.setattr(O, name, fn)
    for pin in pins:
        with pytest.raises((AssertionError, ValueError, np.linalg.LinAlgError)):
            pin()
