"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: entry-wise
brute-force assembly, closed forms (Fourier eigenpairs of the filter),
library routines the oracle does not call (scipy, torch), textbook special
cases (classical multigrid error propagation), and invariants of the method
(positive homogeneity, the one-cycle decomposition of Section 3.2).
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import nmg_inputs as I
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# operators: dense assembly from the definition vs the oracle's structured form
# ---------------------------------------------------------------------------

def brute_2d_operator(taps, n, alpha):
    """A[(i,j),(a,b)] = alpha d_ia d_jb + g_{|i-a|} g_{|j-b|} (Section 4.2), built
    entry by entry, row-major (i, j) -> i*n + j."""
    w = len(taps) - 1
    g = lambda d: taps[abs(d)] if abs(d) <= w else 0.0  # noqa: E731
    A = np.zeros((n * n, n * n))
    for i, j, a, b in itertools.product(range(n), repeat=4):
        A[i * n + j, a * n + b] = alpha * (i == a) * (j == b) + g(i - a) * g(j - b)
    return A


@pytest.mark.parametrize("n,sigma", [(8, 1.0), (12, 2.0)])
def test_2d_apply_matches_bruteforce_assembly(n, sigma):
    taps = I.gaussian_taps(sigma)
    alpha = 1e-2
    H = O.build_hierarchy_2d(taps, n, alpha, 1 if n % 2 else 2)
    A = brute_2d_operator(taps, n, alpha)
    X = np.random.default_rng(0).standard_normal((3, n, n))
    Y = O.apply_level(H, 0, X)
    Yb = (X.reshape(3, -1) @ A.T).reshape(3, n, n)
    assert np.max(np.abs(Y - Yb)) < 1e-14


def test_1d_operator_matches_definition():
    n = 64
    col = I.kernel_column_1d(n, 0.05)
    alpha = 1e-3
    H = O.build_hierarchy_1d(col, alpha, 2)
    h = 1.0 / n
    for i, j in [(0, 0), (3, 7), (63, 0), (10, 40)]:
        ref = h * np.exp(-((i - j) * h) ** 2 / (2 * 0.05 ** 2)) + alpha * (i == j)
        assert abs(H.ops[0][i, j] - ref) < 1e-16


# ---------------------------------------------------------------------------
# transfer operators (Section 2.3; linear interpolation + full weighting)
# ---------------------------------------------------------------------------

def test_prolongation_interpolates_linear_functions():
    nc = 16
    P = O.prolongation(nc)
    J = np.arange(nc)
    coarse = 3.0 + 0.5 * (2 * J)           # samples of f(t) = 3 + 0.5 t at t = 2J
    fine = P @ coarse
    i = np.arange(2 * nc)
    assert np.allclose(fine[:-1], 3.0 + 0.5 * i[:-1], atol=1e-15)
    # last fine point: half of the last coarse value (zero phantom past the end)
    assert abs(fine[-1] - 0.5 * coarse[-1]) < 1e-15
    assert np.allclose(P.sum(axis=1)[:-1], 1.0)


def test_restriction_is_scaled_transpose_and_full_weighting():
    nf = 32
    R = O.restriction(nf)
    P = O.prolongation(nf // 2)
    assert np.array_equal(R, P.T / 2.0)
    for I_ in range(1, nf // 2):
        row = np.zeros(nf)
        row[2 * I_ - 1], row[2 * I_], row[2 * I_ + 1] = 0.25, 0.5, 0.25
        assert np.array_equal(R[I_], row)
    assert R[0, 0] == 0.5 and R[0, 1] == 0.25 and R[0].sum() == 0.75


def test_2d_transfer_is_kronecker():
    n = 8
    H = O.build_hierarchy_2d(I.gaussian_taps(1.0), n, 1e-2, 2)
    P = O.prolongation(n // 2)
    E = np.random.default_rng(1).standard_normal((2, n // 2, n // 2))
    pe = O.prolong(H, 0, E)
    ref = (E.reshape(2, -1) @ np.kron(P, P).T).reshape(2, n, n)
    assert np.max(np.abs(pe - ref)) < 1e-15
    r = np.random.default_rng(2).standard_normal((2, n, n))
    rr = O.restrict(H, 0, r)
    ref = (r.reshape(2, -1) @ (np.kron(P, P).T / 4.0).T).reshape(2, n // 2, n // 2)
    assert np.max(np.abs(rr - ref)) < 1e-15


# ---------------------------------------------------------------------------
# Galerkin hierarchy
# ---------------------------------------------------------------------------

def test_galerkin_2d_equals_dense_RAP():
    n, alpha = 16, 1e-2
    taps = I.gaussian_taps(1.5)
    H = O.build_hierarchy_2d(taps, n, alpha, 3)
    A = brute_2d_operator(taps, n, alpha)
    for l in range(2):
        nf = n >> l
        P = np.kron(O.prolongation(nf // 2), O.prolongation(nf // 2))
        A = (P.T / 4.0) @ A @ P
        M, K = H.ops[l + 1]
        Ak = alpha * np.kron(M, M) + np.kron(K, K)
        assert np.max(np.abs(A - Ak)) < 1e-15
        assert np.max(np.abs(Ak - Ak.T)) < 1e-16
    assert np.max(np.abs(H.coarse - A)) < 1e-15


def test_galerkin_1d_equals_dense_RAP_and_is_symmetric():
    col = I.kernel_column_1d(256)
    H = O.build_hierarchy_1d(col, 1e-3, 3)
    A = H.ops[0]
    for l in range(2):
        nf = A.shape[0]
        P = O.prolongation(nf // 2)
        A = 0.5 * P.T @ A @ P
        assert np.max(np.abs(A - H.ops[l + 1])) < 1e-15
        assert np.max(np.abs(A - A.T)) < 1e-17


@pytest.mark.parametrize("sigma", [1.0, 2.0, 4.0, 8.0])
def test_band_halfwidth_recursion(sigma):
    """K_l is banded with half-width w_{l+1} = floor(w_l / 2) + 1, M_l tridiagonal."""
    taps = I.gaussian_taps(sigma)
    w = len(taps) - 1
    n = 256
    H = O.build_hierarchy_2d(taps, n, 1e-3, 5)
    for l, (M, K) in enumerate(H.ops):
        nz = np.nonzero(np.abs(K) > 0)
        assert np.max(np.abs(nz[0] - nz[1])) == w
        nzm = np.nonzero(np.abs(M) > 0)
        assert np.max(np.abs(nzm[0] - nzm[1])) == (0 if l == 0 else 1)
        w = w // 2 + 1


# ---------------------------------------------------------------------------
# SPD and the coarse solve
# ---------------------------------------------------------------------------

def test_1d_operator_spd_with_lambda_min_at_least_alpha():
    col = I.kernel_column_1d(256)
    alpha = 1e-3
    H = O.build_hierarchy_1d(col, alpha, 3)
    ev = np.linalg.eigvalsh(H.ops[0])
    # the untruncated Gaussian kernel is positive definite (Bochner)
    assert ev.min() >= alpha * (1 - 1e-9)
    for A in H.ops[1:]:
        assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("sigma,alpha", [(2.0, 1e-2), (4.0, 1e-4), (8.0, 1e-3)])
def test_2d_operator_spd(sigma, alpha):
    taps = I.gaussian_taps(sigma)
    n = 64
    H = O.build_hierarchy_2d(taps, n, alpha, 4)
    # lambda(alpha I + K (x) K) = alpha + lambda_i(K) lambda_j(K)
    for M, K in H.ops[:1]:
        lk = np.linalg.eigvalsh(K)
        lam = alpha + np.outer(lk, lk)
        assert lam.min() > 0
    assert np.linalg.eigvalsh(H.coarse).min() > 0


def test_coarse_cholesky_vs_scipy():
    taps = I.gaussian_taps(2.0)
    H = O.build_hierarchy_2d(taps, 128, 1e-2, 5)
    A = H.coarse
    assert A.shape == (64, 64)
    Lsc = sla.cholesky(A, lower=True)
    assert np.max(np.abs(H.chol - Lsc)) < 1e-13 * np.max(np.abs(Lsc))
    y = np.random.default_rng(3).standard_normal((64, 5))
    x = O.cholesky_solve(H.chol, y)
    xl = sla.lu_solve(sla.lu_factor(A), y)
    assert np.max(np.abs(x - xl)) / np.max(np.abs(xl)) < 1e-12


def test_cholesky_rejects_indefinite():
    A = np.eye(4)
    A[2, 2] = -1e-3
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky(A)


# ---------------------------------------------------------------------------
# the output filter F' (Sections 3.2, 3.3): closed-form eigenpairs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [16, 64])
def test_filter_1d_cosine_eigenvectors(n):
    i = np.arange(n)
    for k in range(0, n // 2 + 1):
        v = np.cos(2 * np.pi * k * i / n)[None]
        out = O.spectral_filter(v, 1)
        assert np.max(np.abs(out - np.sqrt(2.0 * k / n) * v)) < 1e-13
        s = np.sin(2 * np.pi * k * i / n)[None]
        out = O.spectral_filter(s, 1)
        assert np.max(np.abs(out - np.sqrt(2.0 * k / n) * s)) < 1e-13


def test_filter_2d_cosine_products_and_special_vectors():
    n = 16
    i = np.arange(n)
    for k1, k2 in [(0, 0), (1, 0), (3, 5), (8, 2), (8, 8), (4, 4)]:
        v = np.outer(np.cos(2 * np.pi * k1 * i / n), np.cos(2 * np.pi * k2 * i / n))[None]
        out = O.spectral_filter(v, 2)
        assert np.max(np.abs(out - np.sqrt(2.0 * max(k1, k2) / n) * v)) < 1e-13
    const = np.ones((1, n, n))
    assert np.max(np.abs(O.spectral_filter(const, 2))) < 1e-14
    alt = np.outer((-1.0) ** i, (-1.0) ** i)[None]
    assert np.max(np.abs(O.spectral_filter(alt, 2) - alt)) < 1e-13


def test_filter_matches_bruteforce_dft():
    """Direct O(n^4) DFT sums with the paper's frequency grid phi_k = (2k-n)pi/n."""
    n = 8
    rng = np.random.default_rng(4)
    h = rng.standard_normal((n, n))
    phi = (2 * np.arange(n) - n) * np.pi / n
    m = np.sqrt(np.maximum(np.abs(phi)[:, None], np.abs(phi)[None, :]) / np.pi)
    out = np.zeros((n, n))
    for a, b in itertools.product(range(n), repeat=2):
        acc = 0j
        for k1, k2 in itertools.product(range(n), repeat=2):
            H_ = sum(h[p, q] * np.exp(-1j * (phi[k1] * p + phi[k2] * q))
                     for p in range(n) for q in range(n))
            acc += m[k1, k2] * H_ * np.exp(1j * (phi[k1] * a + phi[k2] * b))
        out[a, b] = (acc / (n * n)).real
    assert np.max(np.abs(O.spectral_filter(h[None], 2)[0] - out)) < 1e-12


def test_filter_identity_mask():
    h = np.random.default_rng(5).standard_normal((2, 16, 16))
    assert np.max(np.abs(O.spectral_filter(h, 2, mask=np.ones((16, 16))) - h)) < 1e-14


# ---------------------------------------------------------------------------
# CNN smoother vs torch (an independent library), homogeneity
# ---------------------------------------------------------------------------

def test_cnn_2d_matches_torch_conv():
    torch = pytest.importorskip("torch")
    W = I.random_cnn_weights(2, 1, seed=7)[0]
    x = np.random.default_rng(6).standard_normal((3, 20, 20))
    z = torch.tensor(x[:, None])
    for i, (w, b) in enumerate(W):
        z = torch.nn.functional.conv2d(z, torch.tensor(w), torch.tensor(b), padding=1)
        if i < len(W) - 1:
            z = torch.relu(z)
    ref = z[:, 0].numpy()
    out = O.cnn_forward(W, x)
    assert np.max(np.abs(out - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_cnn_1d_matches_torch_conv():
    torch = pytest.importorskip("torch")
    W = I.random_cnn_weights(1, 1, seed=8)[0]
    x = np.random.default_rng(7).standard_normal((4, 37))
    z = torch.tensor(x[:, None])
    for i, (w, b) in enumerate(W):
        z = torch.nn.functional.conv1d(z, torch.tensor(w), torch.tensor(b), padding=2)
        if i < len(W) - 1:
            z = torch.relu(z)
    out = O.cnn_forward(W, x)
    assert np.max(np.abs(out - z[:, 0].numpy())) < 1e-12 * max(1.0, np.max(np.abs(out)))


def test_smoother_is_positively_homogeneous_and_zero_safe():
    W = I.random_cnn_weights(2, 1, seed=9)[0]
    b = np.random.default_rng(8).standard_normal((2, 12, 12))
    h = O.smoother(W, b)
    assert np.max(np.abs(O.smoother(W, 3.7 * b) - 3.7 * h)) < 1e-12 * np.max(np.abs(h))
    assert np.all(O.smoother(W, np.zeros((1, 12, 12))) == 0.0)


# ---------------------------------------------------------------------------
# whole-cycle special cases
# ---------------------------------------------------------------------------

def _zero_weights(dim, nlev):
    W = I.random_cnn_weights(dim, nlev, seed=0)
    return [[(0 * w, 0 * b) for (w, b) in lv] for lv in W]


def test_cycle_with_zero_smoother_is_pure_coarse_correction():
    n, L, alpha = 32, 3, 1e-2
    taps = I.gaussian_taps(1.0)
    H = O.build_hierarchy_2d(taps, n, alpha, L)
    y = np.random.default_rng(9).standard_normal((2, n, n))
    x = O.nmgf(H, _zero_weights(2, L - 1), 0, None, y)
    # dense: P1 P2 A_L^{-1} R2 R1 y with brute-force dense transfers and RAP
    A = brute_2d_operator(taps, n, alpha)
    Ps = [np.kron(O.prolongation((n >> l) // 2), O.prolongation((n >> l) // 2)) for l in range(L - 1)]
    Ac = A
    for P in Ps:
        Ac = (P.T / 4) @ Ac @ P
    Pall = Ps[0] @ Ps[1]
    ref = (Pall @ np.linalg.solve(Ac, (Pall.T / 16.0) @ y.reshape(2, -1).T)).T.reshape(2, n, n)
    assert np.max(np.abs(x - ref)) < 1e-12 * np.max(np.abs(ref))


def test_linear_jacobi_smoother_reproduces_classical_backslash_mg():
    """A one-layer linear 'network' w * b with w = omega / diag(A_l) is weighted
    Jacobi (Section 2.2); with the filter off, s N(b/s) = N(b), and the cycle is
    the classical backslash cycle (Algorithm 1, nu1 = 1, nu2 = 0), whose error
    propagation is the textbook product (I - P A_c^{-1} R A)(I - omega D^{-1} A)."""
    n, L, omega = 64, 2, 0.6
    col = I.kernel_column_1d(n, 0.05)
    H = O.build_hierarchy_1d(col, 1e-2, L)
    A = H.ops[0]
    d = A[0, 0]
    W = [[(np.array([[[0.0, omega / d, 0.0]]]), np.array([0.0]))]]
    P = O.prolongation(n // 2)
    R = P.T / 2
    E = (np.eye(n) - P @ np.linalg.solve(R @ A @ P, R @ A)) @ (np.eye(n) - omega / d * A)
    xtrue = np.random.default_rng(10).standard_normal((3, n))
    y = xtrue @ A.T
    x0 = np.random.default_rng(11).standard_normal((3, n))
    x1 = O.nmgf(H, W, 0, x0, y, filt=False)
    ref = xtrue + (x0 - xtrue) @ E.T
    assert np.max(np.abs(x1 - ref)) < 1e-10 * np.max(np.abs(ref))


def test_single_level_cycle_is_exact_solve():
    n = 8
    taps = I.gaussian_taps(1.0)
    H = O.build_hierarchy_2d(taps, n, 1e-2, 1)
    y = np.random.default_rng(12).standard_normal((2, n, n))
    x = O.nmgf(H, [], 0, None, y)
    A = brute_2d_operator(taps, n, 1e-2)
    ref = np.linalg.solve(A, y.reshape(2, -1).T).T.reshape(2, n, n)
    assert np.max(np.abs(x - ref)) < 1e-12 * np.max(np.abs(ref))


def test_one_cycle_decomposition_identity():
    """With x* = 0, one cycle equals sum_l I_l^1 F'_l(h_l) + I_L^1 (A^(L))^{-1} y_L
    (the decomposition stated in Section 3.2, with the filtered outputs)."""
    n, L = 32, 3
    H = O.build_hierarchy_2d(I.gaussian_taps(1.0), n, 1e-2, L)
    W = I.random_cnn_weights(2, L - 1, seed=13)
    y = np.random.default_rng(14).standard_normal((2, n, n))
    tr = {}
    x = O.nmgf(H, W, 0, None, y, trace=tr)
    total = np.zeros_like(y)
    for l in range(L):
        v = O.spectral_filter(tr["h"][l], 2) if l < L - 1 else tr["x"][l]
        for k in range(l - 1, -1, -1):
            v = O.prolong(H, k, v)
        total += v
    assert np.max(np.abs(x - total)) < 1e-12 * np.max(np.abs(x))


def test_cycle_positive_homogeneity():
    n, L = 32, 3
    H = O.build_hierarchy_2d(I.gaussian_taps(1.0), n, 1e-2, L)
    W = I.random_cnn_weights(2, L - 1, seed=15)
    y = np.random.default_rng(16).standard_normal((2, n, n))
    x = O.nmgf(H, W, 0, None, y)
    x2 = O.nmgf(H, W, 0, None, 2.5 * y)
    assert np.max(np.abs(x2 - 2.5 * x)) < 1e-12 * np.max(np.abs(x2))


def test_cycle_with_initial_guess_is_defect_correction():
    """NMGF(x*, y) = x* + NMGF(0, y - A x*): the identity that makes the
    refinement form (outer residual, inner cycle from zero) the same iteration."""
    n, L = 32, 3
    H = O.build_hierarchy_2d(I.gaussian_taps(1.0), n, 1e-2, L)
    W = I.random_cnn_weights(2, L - 1, seed=17)
    rng = np.random.default_rng(18)
    y = rng.standard_normal((2, n, n))
    xs = rng.standard_normal((2, n, n))
    a = O.nmgf(H, W, 0, xs, y)
    b = xs + O.nmgf(H, W, 0, None, y - O.apply_level(H, 0, xs))
    assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(a))


# ---------------------------------------------------------------------------
# paper's printed closed forms (Section 2.2), golden fixture
# ---------------------------------------------------------------------------

# (the printed Jacobi symbol values pin the oracle's weighted Jacobi step in
# test_oracle_classical.py)


# ---------------------------------------------------------------------------
# final answer of a full solve vs an LU solve
# ---------------------------------------------------------------------------

def test_full_solve_1d_converges_to_lu_solution():
    path = os.path.join(os.path.dirname(os.path.dirname(__file__)),
                        "paper_2603_01064_gb300", "weights", "c1_1d_n256_a1e-3.npz")
    if not os.path.exists(path):
        pytest.skip("trained C1 weights not present")
    z = np.load(path)
    W = [[(z[f"l{l}_w{i}"], z[f"l{l}_b{i}"]) for i in range(3)] for l in range(2)]
    col = I.kernel_column_1d(256)
    H = O.build_hierarchy_1d(col, 1e-3, 3)
    f, _ = I.rhs_1d_sines_steps(256, 4, seed=1001)
    u, cyc, rr = O.solve(H, W, f, rtol=1e-6, max_cycles=60)
    assert np.all(rr <= 1e-6), (cyc, rr)
    ulu = sla.lu_solve(sla.lu_factor(H.ops[0]), f.T).T
    kappa = np.linalg.cond(H.ops[0])
    err = np.linalg.norm(u - ulu, axis=1) / np.linalg.norm(ulu, axis=1)
    assert np.all(err <= kappa * 1e-6)


# ---------------------------------------------------------------------------
# anisotropic regularisation (Section 4.1: A = alpha D + K, D tridiagonal)
# ---------------------------------------------------------------------------

def test_aniso_constant_coefficient_is_dirichlet_laplacian():
    """a = 1 reduces the flux form of -(a u')' to the textbook three-point
    Dirichlet Laplacian tridiag(-1, 2, -1) / h^2."""
    n = 16
    diag, off = I.aniso_regularisation_1d(n, a=lambda z: np.ones_like(z))
    assert np.allclose(diag, 2.0 * n * n, rtol=0, atol=1e-12)
    assert np.allclose(off, -1.0 * n * n, rtol=0, atol=1e-12)


def test_aniso_energy_identity():
    """u^T D u equals the discrete energy sum over the n + 1 cell faces of
    a(face) (u_right - u_left)^2 / h^2, with u = 0 outside the grid: the
    defining property of the conservative form, checked on random u."""
    n = 32
    h = 1.0 / n
    diag, off = I.aniso_regularisation_1d(n)
    D = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    rng = np.random.default_rng(5)
    for _ in range(3):
        u = rng.standard_normal(n)
        up = np.concatenate([[0.0], u, [0.0]])
        faces = 1.0 + 0.5 * np.sin(2 * np.pi * np.arange(n + 1) * h)
        energy = np.sum(faces * np.diff(up) ** 2) / (h * h)
        assert abs(u @ D @ u - energy) <= 1e-12 * energy


def test_aniso_hierarchy_spd_and_galerkin():
    """A_1 = hK + alpha D is the dense sum of its parts; every Galerkin level
    R A P is symmetric positive definite."""
    n, alpha = 64, 1e-5
    col = I.kernel_column_1d(n)
    reg = I.aniso_regularisation_1d(n)
    H = O.build_hierarchy_1d(col, alpha, 3, reg=reg)
    i = np.arange(n)
    T = col[np.abs(i[:, None] - i[None, :])]
    D = np.diag(reg[0]) + np.diag(reg[1], 1) + np.diag(reg[1], -1)
    assert np.abs(H.ops[0] - (T + alpha * D)).max() <= 1e-15 * np.abs(H.ops[0]).max()
    for A in H.ops:
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
        assert np.linalg.eigvalsh(A).min() > 0


def test_full_solve_1d_aniso_converges_to_lu_solution():
    path = os.path.join(os.path.dirname(os.path.dirname(__file__)),
                        "paper_2603_01064_gb300", "weights", "c1a_1d_n256_aniso_a1e-5.npz")
    if not os.path.exists(path):
        pytest.skip("trained anisotropic weights not present")
    z = np.load(path)
    W = [[(z[f"l{l}_w{i}"], z[f"l{l}_b{i}"]) for i in range(3)] for l in range(2)]
    col = I.kernel_column_1d(256)
    H = O.build_hierarchy_1d(col, 1e-5, 3, reg=I.aniso_regularisation_1d(256))
    f, _ = I.rhs_1d_sines_steps(256, 4, seed=1011)
    u, cyc, rr = O.solve(H, W, f, rtol=1e-6, max_cycles=60)
    assert np.all(rr <= 1e-6), (cyc, rr)
    ulu = sla.lu_solve(sla.lu_factor(H.ops[0]), f.T).T
    kappa = np.linalg.cond(H.ops[0])
    err = np.linalg.norm(u - ulu, axis=1) / np.linalg.norm(ulu, axis=1)
    assert np.all(err <= kappa * 1e-6)


# ---------------------------------------------------------------------------
# FNO smoother (Section 3.1, Appendix A; reading R13)
# ---------------------------------------------------------------------------

def _fno_full_mask(n, m):
    """The real-output spectral layer with identity R, written on the full
    (complex) DFT grid: modes k1 in [-m, m-1], k2 in (0, m) and their mirror
    images carry weight 1; on the k2 = 0 column (whose imaginary part the
    real inverse discards) k1 and -k1 each carry half of the retained set."""
    M = np.zeros((n, n))
    kept = lambda k1: (k1 % n) < m or (k1 % n) >= n - m  # noqa: E731
    for k1 in range(n):
        for k2 in range(n):
            if 0 < k2 < m and kept(k1):
                M[k1, k2] += 1.0
            if 0 < (-k2) % n < m and kept(-k1):
                M[k1, k2] += 1.0
            if k2 == 0:
                M[k1, 0] = 0.5 * (kept(k1) + kept(-k1))
    return M


def test_fno_spectral_identity_R_is_full_dft_projection():
    """With R the identity on every retained mode, the spectral layer is the
    projection Re(IDFT(M . DFT(z))) with the full-grid mask above, computed
    here with numpy's complex 2D FFT (the oracle uses the real FFTs)."""
    n, m, c = 16, 3, 2
    rng = np.random.default_rng(11)
    z = rng.standard_normal((2, c, n, n))
    R = np.zeros((2, c, c, m, m), np.complex128)
    for i in range(c):
        R[:, i, i] = 1.0
    got = O.fno_spectral(z, R)
    ref = np.real(np.fft.ifft2(_fno_full_mask(n, m) * np.fft.fft2(z)))
    assert np.abs(got - ref).max() < 1e-13


def test_fno_spectral_single_mode_closed_form():
    """One retained mode (k1, k2) = (1, 2) with R = r (c = 1) maps a cosine of
    that frequency to Re(r) cos - Im(r) sin of the same frequency (the DFT of a
    pure wave is a single pair of spikes), and removes a wave of frequency
    (0, m) along the half-spectrum axis, outside the retained set (while
    (m, 0) keeps half its amplitude: -m is retained on that axis, +m is not)."""
    n, m = 16, 3
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    th = 2 * np.pi * (1 * y + 2 * x) / n
    r = 0.7 - 0.4j
    R = np.zeros((2, 1, 1, m, m), np.complex128)
    R[0, 0, 0, 1, 2] = r      # k1 = 1
    R[1, 0, 0, m - 1, 2] = r  # k1 = n - 1 (the mirror row, same weight)
    z = np.cos(th)[None, None]
    got = O.fno_spectral(z, R)[0, 0]
    assert np.abs(got - (r.real * np.cos(th) - r.imag * np.sin(th))).max() < 1e-13
    R2 = np.ones((2, 1, 1, m, m), np.complex128)
    far = np.cos(2 * np.pi * m * x / n)[None, None]
    assert np.abs(O.fno_spectral(far, R2)).max() < 1e-13
    edge = np.cos(2 * np.pi * m * y / n)[None, None]
    assert np.abs(O.fno_spectral(edge, R2) - 0.5 * edge).max() < 1e-13


def test_fno_without_spectral_part_matches_torch():
    """R = 0: the FNO is lift (1x1 conv) -> [conv + bias, ReLU] x L -> 1x1
    projection, checked against torch.nn.functional.conv2d."""
    torch = pytest.importorskip("torch")
    W = I.random_fno_weights(1, 21, width=4, layers=2, modes=2, ksize=3)[0]
    W["layers"] = [(w, b, 0 * R) for (w, b, R) in W["layers"]]
    x = np.random.default_rng(4).standard_normal((2, 12, 12))
    got = O.fno_forward(W, x)
    F = torch.nn.functional
    t = torch.tensor(x[:, None])
    Wl, bl = W["lift"]
    t = F.conv2d(t, torch.tensor(Wl).view(-1, 1, 1, 1), torch.tensor(bl))
    for w, b, _ in W["layers"]:
        t = torch.relu(F.conv2d(t, torch.tensor(w), torch.tensor(b), padding=1))
    Wp, bp = W["proj"]
    t = F.conv2d(t, torch.tensor(Wp).view(1, -1, 1, 1), torch.tensor(bp))
    assert np.abs(got - t[:, 0].numpy()).max() < 1e-12


def test_fno_smoother_is_positively_homogeneous_in_b():
    """h = N(b / ||b||) ||b||: scaling b by s > 0 scales h by s."""
    W = I.random_fno_weights(1, 5, width=4, layers=2, modes=2)[0]
    b = np.random.default_rng(2).standard_normal((3, 16, 16))
    h1 = O.smoother(W, b)
    h2 = O.smoother(W, 3.5 * b)
    assert np.abs(h2 - 3.5 * h1).max() <= 1e-12 * np.abs(h2).max()


def test_fno_spectral_blocks_act_on_their_own_rows():
    """The two R blocks (k1 in [0, m) and k1 in [n - m, n)) act on their own
    rows of the half spectrum: with R = 1 on block 0 and 0 on block 1, the
    wave cos 2 pi (y + 2x) / n (half-spectrum spike at k1 = 1, k2 = 2) passes
    unchanged and cos 2 pi (-y + 2x) / n (spike at k1 = n - 1) is removed;
    swapping the blocks swaps the outcomes."""
    n, m = 16, 3
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    plus = np.cos(2 * np.pi * (y + 2 * x) / n)[None, None]
    minus = np.cos(2 * np.pi * (-y + 2 * x) / n)[None, None]
    R = np.zeros((2, 1, 1, m, m), np.complex128)
    R[0] = 1.0
    assert np.abs(O.fno_spectral(plus, R) - plus).max() < 1e-13
    assert np.abs(O.fno_spectral(minus, R)).max() < 1e-13
    R = R[::-1].copy()
    assert np.abs(O.fno_spectral(plus, R)).max() < 1e-13
    assert np.abs(O.fno_spectral(minus, R) - minus).max() < 1e-13
