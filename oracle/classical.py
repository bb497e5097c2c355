"""FP64 CPU oracle of the classical comparators of the paper's experiments.

TEST INFRASTRUCTURE ONLY, like nmg_oracle: only the test-suite, the smoke
check and the bench's CPU legs may import it; the CUDA library never calls it.

* Weighted Jacobi (Section 2.2): x <- x + omega D^{-1} (y - A x),
  D = diag(A), applied nu times (SMOOTHING of Algorithm 1).
* The multigrid V-cycle MG(A^(l), x*, y, nu1, nu2, l, L) of Algorithm 1 on the
  same Galerkin hierarchy, transfers and exact coarsest solve as the neural
  cycle; the paper's comparator is the backslash cycle nu1 = 5, nu2 = 0
  (Section 4.1).  omega is not printed for that comparator.  In the model
  problem of Section 2.2, D^{-1} A has its spectrum in (0, 2) and omega = 1/2
  maps the top of it to 1; the reading used here does the same for each
  level's operator: omega_l = 1 / rho_l with rho_l the largest row sum of
  D_l^{-1} |A_l| (a Gershgorin bound on the largest eigenvalue of
  D_l^{-1} A_l).  (A fixed omega = 1/2 diverges on these operators: the
  diagonal of a blur is small against its largest eigenvalue.)
* Conjugate gradients (the comparator of Section 4.2, Table 4), the textbook
  recurrence from x^0 = 0 (or a given guess), stopped per right-hand side
  once the recurred residual satisfies ||r|| / ||f|| <= rtol.
"""
from __future__ import annotations

import numpy as np

from .nmg_oracle import Hierarchy, apply_level, cholesky_solve, prolong, restrict, _norms

__all__ = ["level_diagonal", "jacobi_weight", "jacobi_sweeps", "jacobi_smooth", "mg_cycle",
           "mg_solve", "cg"]


def level_diagonal(H: Hierarchy, l: int) -> np.ndarray:
    """diag(A_l) as an array of the level's vector shape: 1D the diagonal of
    the dense A_l; 2D alpha m_i m_j + k_i k_j with m = diag(M_l), k =
    diag(K_l) (the diagonal of alpha M (x) M + K (x) K)."""
    if H.dim == 1:
        return np.diag(H.ops[l]).copy()
    M, K = H.ops[l]
    m, k = np.diag(M), np.diag(K)
    return H.alpha * np.outer(m, m) + np.outer(k, k)


def jacobi_weight(H: Hierarchy, l: int) -> float:
    """omega_l = 1 / max_i (sum_j |A_l[i, j]|) / A_l[i, i] (see the module
    note).  2D: the row of grid point (i, j) of alpha M (x) M + K (x) K has
    absolute sum alpha |M|_i |M|_j + |K|_i |K|_j (|.|_i the absolute row sums
    of the 1D factors)."""
    if H.dim == 1:
        A = H.ops[l]
        rho = np.max(np.sum(np.abs(A), axis=1) / np.diag(A))
    else:
        M, K = H.ops[l]
        sm, sk = np.sum(np.abs(M), axis=1), np.sum(np.abs(K), axis=1)
        rows = H.alpha * np.outer(sm, sm) + np.outer(sk, sk)
        rho = np.max(rows / level_diagonal(H, l))
    return 1.0 / rho


def jacobi_sweeps(apply, d: np.ndarray, x: np.ndarray, y: np.ndarray, nu: int,
                  omega: float) -> np.ndarray:
    """nu steps of the weighted Jacobi iteration x <- x + omega (y - A x) / d
    for an operator given by its apply function and its diagonal d."""
    x = np.array(x, np.float64)
    for _ in range(nu):
        x = x + omega * (y - apply(x)) / d
    return x


def jacobi_smooth(H: Hierarchy, l: int, x: np.ndarray, y: np.ndarray, nu: int,
                  omega: float | None = None) -> np.ndarray:
    """SMOOTHING(A^(l), x, y, nu) of Algorithm 1 with weighted Jacobi
    (omega None: jacobi_weight(H, l))."""
    w = jacobi_weight(H, l) if omega is None else omega
    return jacobi_sweeps(lambda v: apply_level(H, l, v), level_diagonal(H, l), x, y, nu, w)


def mg_cycle(H: Hierarchy, l: int, xstar, y: np.ndarray, nu1: int = 5, nu2: int = 0,
             omega: float | None = None) -> np.ndarray:
    """MG(A^(l), x*, y, nu1, nu2, l, L) of Algorithm 1, in its order:
      coarsest: x_L = (A^(L))^{-1} y_L
      x = SMOOTHING(A, x*, y, nu1)
      y_{l+1} = I_l^{l+1} (y - A x)
      x = x + I_{l+1}^l MG(A^(l+1), 0, y_{l+1}, ...)
      x = SMOOTHING(A, x, y, nu2)
    xstar None is the zero vector; omega None: the level's jacobi_weight."""
    if l == H.levels - 1:
        B = y.shape[0]
        return cholesky_solve(H.chol, y.reshape(B, -1).T).T.reshape(y.shape)
    x = np.zeros_like(y) if xstar is None else np.array(xstar, np.float64)
    x = jacobi_smooth(H, l, x, y, nu1, omega)
    yc = restrict(H, l, y - apply_level(H, l, x))
    x = x + prolong(H, l, mg_cycle(H, l + 1, None, yc, nu1, nu2, omega))
    return jacobi_smooth(H, l, x, y, nu2, omega)


def mg_solve(H: Hierarchy, f: np.ndarray, rtol: float = 1e-6, max_cycles: int = 1000,
             nu1: int = 5, nu2: int = 0, omega: float | None = None):
    """x^tau = MG(x^{tau-1}, f) from x^0 = 0 until ||f - A x|| / ||f|| <= rtol
    per right-hand side (frozen afterwards, also once the residual is not
    finite).  Returns (u, cycles, relres)."""
    f = np.asarray(f, np.float64)
    u = np.zeros_like(f)
    B = f.shape[0]
    fn = _norms(f)
    fn = np.where(fn > 0, fn, 1.0)
    cycles = np.zeros(B, dtype=np.int64)
    rr = _norms(f - apply_level(H, 0, u)) / fn
    active = rr > rtol
    for _ in range(max_cycles):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        u[idx] = mg_cycle(H, 0, u[idx], f[idx], nu1, nu2, omega)
        cycles[idx] += 1
        rr[idx] = _norms(f[idx] - apply_level(H, 0, u[idx])) / fn[idx]
        active[idx] = (rr[idx] > rtol) & np.isfinite(rr[idx])
    return u, cycles, rr


def cg(H: Hierarchy, f: np.ndarray, rtol: float = 1e-6, max_iters: int = 10000, u0=None):
    """Conjugate gradients on A_1 u = f, per right-hand side:
      r = f - A u, p = r
      repeat: a = (r, r) / (p, A p); u += a p; r -= a A p;
              b = (r_new, r_new) / (r, r); p = r_new + b p
    stopped once ||r|| / ||f|| <= rtol (r the recurred residual).  Returns
    (u, iterations, relres of the recurred residual)."""
    f = np.asarray(f, np.float64)
    B = f.shape[0]
    u = np.zeros_like(f) if u0 is None else np.array(u0, np.float64)
    r = f - apply_level(H, 0, u)
    p = r.copy()
    fn = _norms(f)
    fn = np.where(fn > 0, fn, 1.0)
    rr = np.array([np.dot(r[b].ravel(), r[b].ravel()) for b in range(B)])
    its = np.zeros(B, dtype=np.int64)
    active = np.sqrt(rr) / fn > rtol
    for _ in range(max_iters):
        if not active.any():
            break
        for b in np.nonzero(active)[0]:
            Ap = apply_level(H, 0, p[b:b + 1])[0]
            a = rr[b] / np.dot(p[b].ravel(), Ap.ravel())
            u[b] = u[b] + a * p[b]
            r[b] = r[b] - a * Ap
            rr_new = np.dot(r[b].ravel(), r[b].ravel())
            p[b] = r[b] + (rr_new / rr[b]) * p[b]
            rr[b] = rr_new
            its[b] += 1
            active[b] = np.sqrt(rr[b]) / fn[b] > rtol
    return u, its, np.sqrt(rr) / fn
