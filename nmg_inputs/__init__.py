"""Seeded synthetic inputs for the neural multigrid solve.

This module is shared by the CPU oracle, the tests, the bench and the offline
smoother trainer. It holds only problem *data*: the discretised kernel that
defines the operator (Eq. (1) discretised on a uniform mesh, Section 2.1) and
seeded right-hand sides. It contains none of the multigrid method's
arithmetic (no Galerkin products, smoothers, filters or solves).

Every generator takes an explicit integer seed and uses numpy's PCG64.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "gaussian_taps",
    "kernel_column_1d",
    "blur_1d",
    "blur_2d",
    "rhs_1d_sines_steps",
    "rhs_2d_ellipses_grf",
    "rhs_2d_waves_rects",
    "random_cnn_weights",
    "CONFIGS",
]


# ---------------------------------------------------------------------------
# operator data
# ---------------------------------------------------------------------------

def gaussian_taps(sigma: float) -> np.ndarray:
    """Normalised 1D Gaussian point-spread taps g_0..g_w with w = ceil(4 sigma).

    The 2D operator of Section 4.2 is alpha I (x) I + K (x) K with K the 1D
    convolution matrix; K is Toeplitz with K[i, j] = g_{|i-j|} for
    |i-j| <= w and zero otherwise (zero boundary, truncated at 4 sigma,
    taps summing to one over -w..w).
    """
    w = int(math.ceil(4.0 * sigma))
    j = np.arange(-w, w + 1, dtype=np.float64)
    e = np.exp(-(j * j) / (2.0 * sigma * sigma))
    e /= e.sum()
    return np.ascontiguousarray(e[w:])  # g_0 .. g_w


def kernel_column_1d(n: int, width: float = 0.05) -> np.ndarray:
    """First column of h*K for the 1D Fredholm problem (Eq. (1), Section 2.1).

    Midpoint rule on n cells of [0, 1]: (hK)[i, j] = h * k((i - j) h) with
    k(t) = exp(-t^2 / (2 width^2)).  The matrix is symmetric Toeplitz, so the
    first column t_d = h k(d h), d = 0..n-1, defines it.
    """
    h = 1.0 / n
    d = np.arange(n, dtype=np.float64) * h
    return h * np.exp(-(d * d) / (2.0 * width * width))


def aniso_coefficient(z: np.ndarray) -> np.ndarray:
    """Coefficient a(z) = 1 + 0.5 sin(2 pi z) of the anisotropic
    regularisation of Section 4.1 (R(u) = -(a u')')."""
    return 1.0 + 0.5 * np.sin(2.0 * np.pi * z)


def aniso_regularisation_1d(n: int, a=aniso_coefficient):
    """Tridiagonal D of the anisotropic regularisation (Section 4.1, A = alpha
    D + K), as (diag, off): the conservative three-point form of -(a u')' on
    the n midpoint cells of [0, 1] with u = 0 outside, coefficients at the
    cell faces z = i h:
        (D u)_i = (a(ih) (u_i - u_{i-1}) - a((i+1)h) (u_{i+1} - u_i)) / h^2.
    diag has n entries, off the n - 1 sub/super-diagonal entries."""
    h = 1.0 / n
    faces = a(np.arange(n + 1, dtype=np.float64) * h)  # a(0), a(h), ..., a(1)
    diag = (faces[:-1] + faces[1:]) / (h * h)
    off = -faces[1:-1] / (h * h)
    return diag, off


def blur_1d(u: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Data model of the 1D problem: the discrete blur (hK) u, u of shape [B, n]."""
    n = u.shape[-1]
    i = np.arange(n)
    T = col[np.abs(i[:, None] - i[None, :])]
    return u @ T.T


def _conv_same_axis(x: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """Zero-boundary symmetric convolution along one axis (data model only)."""
    w = len(taps) - 1
    full = np.concatenate([taps[::-1], taps[1:]])
    x = np.moveaxis(x, axis, -1)
    n = x.shape[-1]
    xp = np.zeros(x.shape[:-1] + (n + 2 * w,))
    xp[..., w:w + n] = x
    out = np.zeros_like(x)
    for k in range(2 * w + 1):
        out += full[k] * xp[..., k:k + n]
    return np.moveaxis(out, -1, axis)


def blur_2d(u: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """Data model of the 2D problem: separable PSF blur K U K^T, u of shape [B, n, n]."""
    return _conv_same_axis(_conv_same_axis(u, taps, -1), taps, -2)


# ---------------------------------------------------------------------------
# right-hand sides (the paper uses randomly generated right-hand sides)
# ---------------------------------------------------------------------------

def _add_noise(clean: np.ndarray, rng: np.random.Generator, level: float) -> np.ndarray:
    axes = tuple(range(1, clean.ndim))
    rms = np.sqrt(np.mean(clean * clean, axis=axes, keepdims=True))
    return clean + level * rms * rng.standard_normal(clean.shape)


def rhs_1d_sines_steps(n: int, batch: int, seed: int, width: float = 0.05,
                       noise: float = 0.01):
    """1D right-hand sides f = (hK) u_true + 1% Gaussian noise.

    u_true(t) = sum_{j=1..8} a_j sin(2 pi k_j t + phi_j) + sum_{s=1,2} c_s 1[t >= tau_s]
    with a, c ~ U(-1, 1), k ~ U{1..16}, phi ~ U(0, 2 pi), tau ~ U(0.1, 0.9).
    Returns (f, u_true), both float64 [batch, n].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = (np.arange(n) + 0.5) / n
    u = np.zeros((batch, n))
    for b in range(batch):
        a = rng.uniform(-1, 1, 8)
        k = rng.integers(1, 17, 8)
        ph = rng.uniform(0, 2 * np.pi, 8)
        for j in range(8):
            u[b] += a[j] * np.sin(2 * np.pi * k[j] * t + ph[j])
        c = rng.uniform(-1, 1, 2)
        tau = rng.uniform(0.1, 0.9, 2)
        for s in range(2):
            u[b] += c[s] * (t >= tau[s])
    f = _add_noise(blur_1d(u, kernel_column_1d(n, width)), rng, noise)
    return f, u


def rhs_2d_ellipses_grf(n: int, batch: int, seed: int, sigma: float,
                        corr: float = 8.0, noise: float = 0.01):
    """2D piecewise-smooth right-hand sides: 5-10 random ellipses (intensity
    U(0, 1)) plus a Gaussian random field (white noise smoothed with a
    Gaussian of correlation length `corr` px, scaled to std 0.1), blurred by
    the PSF with zero boundary, plus 1% Gaussian noise.
    Returns (f, u_true), float64 [batch, n, n].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.meshgrid((np.arange(n) + 0.5) / n, (np.arange(n) + 0.5) / n, indexing="ij")
    grf_taps = gaussian_taps(corr / 2.0)
    u = np.zeros((batch, n, n))
    for b in range(batch):
        for _ in range(int(rng.integers(5, 11))):
            cy, cx = rng.uniform(0.1, 0.9, 2)
            ry, rx = rng.uniform(0.03, 0.3, 2)
            th = rng.uniform(0, np.pi)
            dy, dx = yy - cy, xx - cx
            p = (np.cos(th) * dx + np.sin(th) * dy) / rx
            q = (-np.sin(th) * dx + np.cos(th) * dy) / ry
            u[b] += rng.uniform(0, 1) * ((p * p + q * q) <= 1.0)
        g = blur_2d(rng.standard_normal((1, n, n)), grf_taps)[0]
        u[b] += 0.1 * g / max(np.std(g), 1e-30)
    f = _add_noise(blur_2d(u, gaussian_taps(sigma)), rng, noise)
    return f, u


def rhs_2d_waves_rects(n: int, batch: int, seed: int, sigma: float, noise: float = 0.01):
    """2D analogue of the 1D generator: 8 random plane waves
    a sin(2 pi (kx x + ky y) + phi) plus 2 random axis-aligned rectangles of
    random height, blurred by the PSF, plus 1% Gaussian noise.
    Returns (f, u_true), float64 [batch, n, n].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.meshgrid((np.arange(n) + 0.5) / n, (np.arange(n) + 0.5) / n, indexing="ij")
    u = np.zeros((batch, n, n))
    for b in range(batch):
        for _ in range(8):
            a = rng.uniform(-1, 1)
            kx, ky = rng.integers(-16, 17, 2)
            ph = rng.uniform(0, 2 * np.pi)
            u[b] += a * np.sin(2 * np.pi * (kx * xx + ky * yy) + ph)
        for _ in range(2):
            y0, x0 = rng.uniform(0.0, 0.8, 2)
            hy, hx = rng.uniform(0.05, 0.4, 2)
            u[b] += rng.uniform(-1, 1) * ((yy >= y0) & (yy < y0 + hy) & (xx >= x0) & (xx < x0 + hx))
    f = _add_noise(blur_2d(u, gaussian_taps(sigma)), rng, noise)
    return f, u


# ---------------------------------------------------------------------------
# smoother weights for parity tests (untrained, seeded)
# ---------------------------------------------------------------------------

def random_cnn_weights(dim: int, nlevels: int, seed: int, width: int | None = None,
                       layers: int | None = None, ksize: int | None = None,
                       scale: float = 1.0):
    """Seeded He-style random CNN weights in PyTorch Conv layout.

    Returns a list (one entry per smoother level) of lists of (W, b) with
    W of shape [Cout, Cin, k] (1D) or [Cout, Cin, k, k] (2D).
    Defaults: 1D 3 layers, width 16, k 5; 2D 4 layers, width 32, 3x3.
    """
    if width is None:
        width = 16 if dim == 1 else 32
    if layers is None:
        layers = 3 if dim == 1 else 4
    if ksize is None:
        ksize = 5 if dim == 1 else 3
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(nlevels):
        lv = []
        for li in range(layers):
            cin = 1 if li == 0 else width
            cout = 1 if li == layers - 1 else width
            shape = (cout, cin) + (ksize,) * dim
            fan_in = cin * ksize ** dim
            W = scale * rng.standard_normal(shape) * math.sqrt(2.0 / fan_in)
            b = 0.1 * scale * rng.standard_normal(cout)
            lv.append((W, b))
        out.append(lv)
    return out


# ---------------------------------------------------------------------------
# the five workload descriptions (sizes, operators, precisions)
# ---------------------------------------------------------------------------

CONFIGS = {
    "c1_1d_fp64": dict(dim=1, n=256, levels=3, alpha=1e-3, width=0.05, batch=16,
                       precision="fp64", rhs_seed=1001),
    "c2_2d_fp32": dict(dim=2, n=128, levels=5, alpha=1e-2, sigma=2.0, batch=256,
                       precision="fp32", rhs_seed=1002),
    "c3_2d_bf16": dict(dim=2, n=512, levels=7, alphas=(1e-4, 1e-3, 1e-2, 1e-1), sigma=4.0,
                       batch=64, precision="bf16_refine", rhs_seed=1003),
}


def random_fno_weights(nlevels: int, seed: int, width: int = 8, layers: int = 2,
                       modes: int = 4, ksize: int = 3):
    """Seeded random weights of the 2D FNO smoother (Appendix A: lift 1 -> c,
    `layers` Fourier layers with a ksize x ksize W term and complex R on
    `modes` modes per axis, projection c -> 1), one dict per level:
    dict(lift=(Wl [c], bl [c]), layers=[(W [c, c, k, k], b [c],
    R [2, c, c, m, m] complex)], proj=(Wp [c], bp [1])).  He-style scales
    keep the activations O(1)."""
    rng = np.random.default_rng(seed)
    c, m, k = width, modes, ksize
    out = []
    for _ in range(nlevels):
        lift = (rng.standard_normal(c), 0.1 * rng.standard_normal(c))
        lay = []
        for _ in range(layers):
            W = rng.standard_normal((c, c, k, k)) * math.sqrt(1.0 / (c * k * k))
            b = 0.1 * rng.standard_normal(c)
            R = (rng.standard_normal((2, c, c, m, m)) + 1j * rng.standard_normal((2, c, c, m, m)))
            lay.append((W, b, R * math.sqrt(1.0 / c)))
        proj = (rng.standard_normal(c) * math.sqrt(1.0 / c), 0.1 * rng.standard_normal(1))
        out.append(dict(lift=lift, layers=lay, proj=proj))
    return out
