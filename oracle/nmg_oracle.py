"""FP64 CPU oracle of the neural multigrid solve (Algorithms 3 and 4).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
bench's CPU-baseline leg may import this module.  The CUDA library never
calls it and shares no code with it: the two are compared, never combined.

Everything is plain float64 numpy, written to follow the paper step by step:

* operators are assembled densely from their definitions (Section 2.1,
  Eq. (10) in 1D and the Kronecker form of Section 4.2 in 2D);
* the transfer operators are explicit dense matrices (Section 2.3);
* coarse operators are the Galerkin products R A P (Algorithm 1, step
  A^(l+1) <- I_l^{l+1} A^(l) I_{l+1}^l);
* the coarsest system is solved with a hand-written dense Cholesky;
* the smoother is the CNN applied by a direct convolution sum, or the FNO of
  Appendix A (spectral part by numpy's real FFTs);
* the output filter is Re(IDFT(m' . DFT(h))) (Sections 3.2 and 3.3) using
  numpy's FFT as a library primitive;
* the cycle is NMGF1d / NMGF2d exactly as Algorithms 3 and 4 list it, and the
  outer iteration is x^tau = NMGF(x^{tau-1}, y) from x^0 = 0 (Section 3.2).

Readings of the paper where it is silent or garbled (all listed in the
design notes of the repository):
  R1  transfer operators: linear interpolation with coarse node J at fine
      node 2J, fine 2J+1 the mean of J and J+1 (zero past the end);
      restriction is full weighting R = P^T / 2 per axis.
  R2  mask: m_l(phi) = sqrt(|phi| / (pi/2^{l-1})) (the printed formula has
      no absolute value), discretised on the level grid so every level uses
      the same local symbol sqrt(|omega| / pi), 2D uses max(|w1|, |w2|).
  R3  the filter is periodic (a DFT on the level grid), forward DFT
      unnormalised and inverse scaled by 1/n per axis.
  R4  ||b|| = 0 gives h = 0.
  R5  smoothers sit on levels 1..L-1 and the coarsest level L has the
      exact solve.
  R13 FNO: the retained modes are the half spectrum of the real 2D DFT with
      k1 in [0, m) and [n - m, n), k2 in [0, m) (the FNO the paper cites);
      sigma = ReLU after every Fourier layer; the lift and projection are
      pointwise affine maps.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "prolongation", "restriction", "toeplitz_from_column", "banded_toeplitz",
    "Hierarchy", "build_hierarchy_1d", "build_hierarchy_2d",
    "cholesky", "cholesky_solve", "apply_level", "cnn_forward", "fno_spectral", "fno_forward",
    "smoother",
    "filter_mask", "spectral_filter", "restrict", "prolong", "nmgf", "relres", "solve",
]


# ---------------------------------------------------------------------------
# transfer operators (Section 2.3; reading R1)
# ---------------------------------------------------------------------------

def prolongation(nc: int) -> np.ndarray:
    """Dense 1D linear interpolation I_{l+1}^l of shape [2 nc, nc]."""
    nf = 2 * nc
    P = np.zeros((nf, nc))
    for J in range(nc):
        P[2 * J, J] = 1.0
        P[2 * J + 1, J] = 0.5
        if 2 * J - 1 >= 0:
            P[2 * J - 1, J] = 0.5
    return P


def restriction(nf: int) -> np.ndarray:
    """Dense 1D full weighting I_l^{l+1} = P^T / 2 of shape [nf/2, nf]."""
    return prolongation(nf // 2).T / 2.0


# ---------------------------------------------------------------------------
# fine-grid operators (Section 2.1, Eq. (10), Section 4.2)
# ---------------------------------------------------------------------------

def toeplitz_from_column(col: np.ndarray) -> np.ndarray:
    """Symmetric Toeplitz matrix T[i, j] = col[|i - j|]."""
    n = len(col)
    T = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            T[i, j] = col[abs(i - j)]
    return T


def banded_toeplitz(taps: np.ndarray, n: int) -> np.ndarray:
    """Symmetric banded Toeplitz K[i, j] = taps[|i-j|] if |i-j| <= w else 0."""
    w = len(taps) - 1
    K = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - w), min(n, i + w + 1)):
            K[i, j] = taps[abs(i - j)]
    return K


class Hierarchy:
    """Level operators of the Galerkin hierarchy.

    dim == 1: ops[l] = dense A_l (n_l x n_l).
    dim == 2: ops[l] = (M_l, K_l) with A_l = alpha M_l (x) M_l + K_l (x) K_l.
    coarse = dense A_L, chol = its Cholesky factor (lower).
    Index 0 is the finest level (the paper's l = 1).
    """

    def __init__(self, dim, n, levels, alpha, ops, coarse):
        self.dim = dim
        self.n = n
        self.levels = levels
        self.alpha = alpha
        self.ops = ops
        self.coarse = coarse
        self.chol = cholesky(coarse)

    def size(self, l: int) -> int:
        return self.n >> l


def build_hierarchy_1d(col: np.ndarray, alpha: float, levels: int, reg=None) -> Hierarchy:
    """1D: A_1 = hK + alpha I (Eq. (10) with the kernel column given by the
    midpoint rule), A_{l+1} = R A_l P (Algorithm 3, Galerkin).  With reg =
    (diag, off), the anisotropic case of Section 4.1: A_1 = hK + alpha D with
    D the symmetric tridiagonal matrix of those diagonals."""
    n = len(col)
    assert n % (1 << (levels - 1)) == 0
    if reg is None:
        D = np.eye(n)
    else:
        diag, off = reg
        D = np.diag(np.asarray(diag, dtype=np.float64)) + np.diag(off, 1) + np.diag(off, -1)
    A = toeplitz_from_column(col) + alpha * D
    ops = [A]
    for _ in range(levels - 1):
        nf = A.shape[0]
        A = restriction(nf) @ A @ prolongation(nf // 2)
        ops.append(A)
    return Hierarchy(1, n, levels, alpha, ops, ops[-1].copy())


def build_hierarchy_2d(taps: np.ndarray, n: int, alpha: float, levels: int) -> Hierarchy:
    """2D: A_1 = alpha I (x) I + K (x) K (Section 4.2); since
    (R(x)R)(alpha M(x)M + K(x)K)(P(x)P) = alpha (RMP)(x)(RMP) + (RKP)(x)(RKP),
    the Galerkin operator of Algorithm 4 stays in this form with
    M_{l+1} = R M_l P and K_{l+1} = R K_l P."""
    assert n % (1 << (levels - 1)) == 0
    M = np.eye(n)
    K = banded_toeplitz(taps, n)
    ops = [(M, K)]
    for _ in range(levels - 1):
        nf = M.shape[0]
        R, P = restriction(nf), prolongation(nf // 2)
        M = R @ M @ P
        K = R @ K @ P
        ops.append((M, K))
    Mc, Kc = ops[-1]
    coarse = alpha * np.kron(Mc, Mc) + np.kron(Kc, Kc)
    return Hierarchy(2, n, levels, alpha, ops, coarse)


# ---------------------------------------------------------------------------
# coarsest solve (Algorithm 3/4: x_L = (A^(L))^{-1} y_L), dense Cholesky
# ---------------------------------------------------------------------------

def cholesky(A: np.ndarray) -> np.ndarray:
    """Textbook column Cholesky A = L L^T; raises if A is not SPD."""
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        d = A[j, j] - np.dot(L[j, :j], L[j, :j])
        if not d > 0.0:
            raise np.linalg.LinAlgError("coarse operator is not positive definite")
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return L


def cholesky_solve(L: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Solve L L^T x = y by forward then back substitution; y is [m] or [m, B]."""
    n = L.shape[0]
    z = np.array(y, dtype=np.float64, copy=True)
    for i in range(n):
        z[i] = (z[i] - L[i, :i] @ z[:i]) / L[i, i]
    x = z
    for i in range(n - 1, -1, -1):
        x[i] = (x[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


# ---------------------------------------------------------------------------
# level operator, transfers on batches
# ---------------------------------------------------------------------------

def apply_level(H: Hierarchy, l: int, x: np.ndarray) -> np.ndarray:
    """A_l x for a batch: 1D x [B, n_l]; 2D x [B, n_l, n_l] with
    Mat(A_l Vec(X)) = alpha M X M^T + K X K^T (Section 3.3, Vec/Mat)."""
    if H.dim == 1:
        return x @ H.ops[l].T
    M, K = H.ops[l]
    return H.alpha * (M @ x @ M.T) + (K @ x @ K.T)


def restrict(H: Hierarchy, l: int, r: np.ndarray) -> np.ndarray:
    """I_l^{l+1} applied to a batch of level-l vectors (2D: R (x) R)."""
    R = restriction(H.size(l))
    if H.dim == 1:
        return r @ R.T
    return R @ r @ R.T


def prolong(H: Hierarchy, l: int, e: np.ndarray) -> np.ndarray:
    """I_{l+1}^l applied to a batch of level-(l+1) vectors (2D: P (x) P)."""
    P = prolongation(H.size(l + 1))
    if H.dim == 1:
        return e @ P.T
    return P @ e @ P.T


# ---------------------------------------------------------------------------
# neural smoother (Section 3.2: h = N(b / ||b||) ||b||), CNN by direct sums
# ---------------------------------------------------------------------------

def _conv_same(x: np.ndarray, W: np.ndarray, bias: np.ndarray) -> np.ndarray:
    """Cross-correlation with zero 'same' padding, PyTorch Conv semantics:
    out[b, o, p] = bias[o] + sum_{c, t} W[o, c, t] x[b, c, p + t - k//2].
    x is [B, Cin, n] (1D) or [B, Cin, n, n] (2D).  The channel sum of each
    tap is one matrix product (numpy's BLAS)."""
    dim = W.ndim - 2
    k = W.shape[-1]
    p = k // 2
    B = x.shape[0]
    n = x.shape[2]
    Cout = W.shape[0]
    if dim == 1:
        xp = np.pad(x, ((0, 0), (0, 0), (p, p)))
        out = np.broadcast_to(bias[None, :, None], (B, Cout, n)).copy()
        for t in range(k):
            out += np.einsum("oc,bcn->bon", W[:, :, t], xp[:, :, t:t + n], optimize=True)
        return out
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p)))
    out = np.broadcast_to(bias[None, :, None, None], (B, Cout, n, n)).copy()
    for ty in range(k):
        for tx in range(k):
            out += np.einsum("oc,bcij->boij", W[:, :, ty, tx], xp[:, :, ty:ty + n, tx:tx + n],
                             optimize=True)
    return out


def cnn_forward(weights, x: np.ndarray) -> np.ndarray:
    """N_theta(x): conv, ReLU, ..., conv (no activation after the last layer).
    weights = [(W, b), ...]; x is [B, n] (1D) or [B, n, n] (2D)."""
    z = x[:, None]
    nl = len(weights)
    for i, (W, b) in enumerate(weights):
        z = _conv_same(z, np.asarray(W, np.float64), np.asarray(b, np.float64))
        if i < nl - 1:
            z = np.maximum(z, 0.0)
    return z[:, 0]


# ---------------------------------------------------------------------------
# FNO smoother (Section 3.1, Appendix A): lift, Fourier layers, projection
# ---------------------------------------------------------------------------

def fno_spectral(z: np.ndarray, R: np.ndarray) -> np.ndarray:
    """DFT^{-1}(R . DFT(z)) of one Fourier layer (Appendix A): R acts only on
    the first m low-frequency modes per axis (reading R13: the half spectrum
    of a real 2D signal, k1 in [0, m) and [n - m, n), k2 in [0, m)) and the
    other modes are zeroed.  z is [B, c, n, n] real, R is [2, c_in, c_out, m,
    m] complex (block 0: k1 = 0..m-1, block 1: k1 = n-m..n-1).  The DFTs are
    numpy's real FFTs (a library primitive)."""
    B, c, n, _ = z.shape
    m = R.shape[-1]
    Z = np.fft.rfft2(z)  # [B, c, n, n/2 + 1]
    Y = np.zeros((B, R.shape[2], n, n // 2 + 1), dtype=np.complex128)
    Y[:, :, :m, :m] = np.einsum("bixy,ioxy->boxy", Z[:, :, :m, :m], R[0])
    Y[:, :, n - m:, :m] = np.einsum("bixy,ioxy->boxy", Z[:, :, n - m:, :m], R[1])
    return np.fft.irfft2(Y, s=(n, n))


def fno_forward(weights, x: np.ndarray) -> np.ndarray:
    """N_theta(x) of the FNO of Appendix A on [B, n, n]: a pointwise lift
    1 -> c, L Fourier layers z <- sigma(DFT^{-1}(R . DFT(z)) + W z + B) with
    W a 'same' convolution and sigma = ReLU (reading R13), then a pointwise
    projection c -> 1.  weights = dict(lift=(Wl [c], bl [c]),
    layers=[(W [c, c, k, k], b [c], R [2, c, c, m, m] complex), ...],
    proj=(Wp [c], bp [1]))."""
    Wl, bl = (np.asarray(a, np.float64) for a in weights["lift"])
    z = Wl[None, :, None, None] * x[:, None] + bl[None, :, None, None]
    for W, b, R in weights["layers"]:
        z = np.maximum(_conv_same(z, np.asarray(W, np.float64), np.asarray(b, np.float64)) +
                       fno_spectral(z, np.asarray(R, np.complex128)), 0.0)
    Wp, bp = (np.asarray(a, np.float64) for a in weights["proj"])
    return np.einsum("c,bcij->bij", Wp, z) + bp[0]


def _norms(v: np.ndarray) -> np.ndarray:
    return np.sqrt(np.sum(v.reshape(v.shape[0], -1) ** 2, axis=1))


def smoother(weights, b: np.ndarray) -> np.ndarray:
    """h = N(b / ||b||_2) ||b||_2 per right-hand side (Algorithm 3/4); h = 0
    where ||b|| = 0 (reading R4)."""
    s = _norms(b)
    shape = (-1,) + (1,) * (b.ndim - 1)
    safe = np.where(s > 0, s, 1.0).reshape(shape)
    net = fno_forward if isinstance(weights, dict) else cnn_forward
    h = net(weights, b / safe) * safe
    return np.where(s.reshape(shape) > 0, h, 0.0)


# ---------------------------------------------------------------------------
# output filter F'_l (Sections 3.2, 3.3; readings R2, R3)
# ---------------------------------------------------------------------------

def filter_mask(n: int, dim: int) -> np.ndarray:
    """m'_l on the DFT bins of an n-point level grid: bin j has angular
    frequency omega_j = 2 pi j / n folded into [-pi, pi]; the local symbol is
    sqrt(|omega| / pi) in 1D and sqrt(max(|omega_1|, |omega_2|) / pi) in 2D."""
    j = np.arange(n)
    w = 2.0 * np.pi * np.minimum(j, n - j) / n
    if dim == 1:
        return np.sqrt(w / np.pi)
    return np.sqrt(np.maximum(w[:, None], w[None, :]) / np.pi)


def spectral_filter(h: np.ndarray, dim: int, mask: np.ndarray | None = None) -> np.ndarray:
    """F'(h) = Re(IDFT(m' . DFT(h))) per right-hand side."""
    n = h.shape[-1]
    if mask is None:
        mask = filter_mask(n, dim)
    if dim == 1:
        return np.real(np.fft.ifft(mask[None] * np.fft.fft(h, axis=-1), axis=-1))
    return np.real(np.fft.ifft2(mask[None] * np.fft.fft2(h, axes=(-2, -1)), axes=(-2, -1)))


# ---------------------------------------------------------------------------
# the cycle (Algorithm 3 in 1D, Algorithm 4 in 2D; Algorithm 2 with filt=False)
# ---------------------------------------------------------------------------

def nmgf(H: Hierarchy, weights, l: int, xstar, y: np.ndarray, filt: bool = True,
         trace: dict | None = None) -> np.ndarray:
    """One neural multigrid cycle at level l (0-based) with initial guess
    xstar (None means the zero vector) and right-hand side y.

    Steps, in the order the algorithms list them:
      coarsest: x_L = (A^(L))^{-1} y_L
      b = y - A x*;  h = N(b/||b||)||b||;  x = x* + F'(h)
      y_{l+1} = I_l^{l+1} (y - A x)
      x = x + I_{l+1}^l NMGF(0, y_{l+1}, l+1)
    """
    if l == H.levels - 1:
        B = y.shape[0]
        ys = y.reshape(B, -1).T
        x = cholesky_solve(H.chol, ys).T.reshape(y.shape)
        if trace is not None:
            trace.setdefault("x", {})[l] = x.copy()
        return x
    if xstar is None:
        b = y.copy()
        xs = np.zeros_like(y)
    else:
        xs = xstar
        b = y - apply_level(H, l, xs)
    h = smoother(weights[l], b)
    x = xs + (spectral_filter(h, H.dim) if filt else h)
    ycoarse = restrict(H, l, y - apply_level(H, l, x))
    if trace is not None:
        trace.setdefault("b", {})[l] = b.copy()
        trace.setdefault("h", {})[l] = h.copy()
        trace.setdefault("xs", {})[l] = x.copy()
        trace.setdefault("y", {})[l + 1] = ycoarse.copy()
    e = nmgf(H, weights, l + 1, None, ycoarse, filt, trace)
    x = x + prolong(H, l, e)
    if trace is not None:
        trace.setdefault("x", {})[l] = x.copy()
    return x


def relres(H: Hierarchy, f: np.ndarray, u: np.ndarray) -> np.ndarray:
    """||f - A u|| / ||f|| per right-hand side."""
    r = f - apply_level(H, 0, u)
    fn = _norms(f)
    return _norms(r) / np.where(fn > 0, fn, 1.0)


def solve(H: Hierarchy, weights, f: np.ndarray, rtol: float = 1e-6, max_cycles: int = 100,
          filt: bool = True, u0: np.ndarray | None = None):
    """Outer iteration x^tau = NMGF(x^{tau-1}, f) from x^0 = 0 (Section 3.2),
    stopped per right-hand side once ||f - A x|| / ||f|| <= rtol.

    Returns (u, cycles [B], relres [B]); a right-hand side that meets the
    tolerance is frozen (no further cycles are applied to it)."""
    f = np.asarray(f, np.float64)
    u = np.zeros_like(f) if u0 is None else np.array(u0, np.float64)
    B = f.shape[0]
    cycles = np.zeros(B, dtype=np.int64)
    rr = relres(H, f, u)
    active = rr > rtol
    for _ in range(max_cycles):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        u[idx] = nmgf(H, weights, 0, u[idx], f[idx], filt)
        cycles[idx] += 1
        rr[idx] = relres(H, f[idx], u[idx])
        active[idx] = rr[idx] > rtol
    return u, cycles, rr
