"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the FP64 oracle (on the CPU, by replacing
one of its functions for the duration of the test) -- a dropped term, a
wrong scale, sign or index, a flipped kernel, a missing normalisation -- and
checks that the named pins of ``test_oracle_pins.py`` then fail.  The
unmodified oracle passes the same pins in that file.
"""
import numpy as np
import pytest

import nmg_inputs as I
import oracle as O
from oracle import nmg_oracle as NO
import test_inputs as TI
import test_oracle_pins as P

CAUGHT = (AssertionError, ValueError, np.linalg.LinAlgError)


def _plant(monkeypatch, name, fn):
    """Replace oracle function `name` in the module (its internal callers)
    and in the package namespace (the pins' callers)."""
    monkeypatch.setattr(NO, name, fn)
    monkeypatch.setattr(O, name, fn, raising=False)


_prolongation = NO.prolongation
_restriction = NO.restriction
_filter_mask = NO.filter_mask
_conv_same = NO._conv_same
_apply_level = NO.apply_level
_fno_spectral = NO.fno_spectral


def restriction_missing_half(nf):
    return _prolongation(nf // 2).T  # P^T instead of P^T / 2


def prolongation_copies_last_point(nc):
    Pm = _prolongation(nc)
    Pm[2 * nc - 1, nc - 1] = 1.0  # constant extension instead of the zero phantom
    return Pm


def mask_without_sqrt(n, dim):
    return _filter_mask(n, dim) ** 2  # |omega| / pi instead of its square root


def mask_min_instead_of_max(n, dim):
    if dim == 1:
        return _filter_mask(n, 1)
    j = np.arange(n)
    w = 2.0 * np.pi * np.minimum(j, n - j) / n
    return np.sqrt(np.minimum(w[:, None], w[None, :]) / np.pi)


def mask_on_unshifted_bins(n, dim):
    # the symbol sampled at phi_k = (2k - n) pi / n but applied to DFT bin k
    # without the shift that puts frequency 0 at bin 0
    phi = np.abs((2 * np.arange(n) - n) * np.pi / n)
    if dim == 1:
        return np.sqrt(phi / np.pi)
    return np.sqrt(np.maximum(phi[:, None], phi[None, :]) / np.pi)


def conv_flipped_kernel(x, W, bias):
    # true convolution instead of PyTorch's cross-correlation
    return _conv_same(x, np.flip(W, axis=tuple(range(2, W.ndim))).copy(), bias)


def cnn_relu_after_last_layer(weights, x):
    z = x[:, None]
    for W, b in weights:
        z = np.maximum(_conv_same(z, np.asarray(W, np.float64), np.asarray(b, np.float64)), 0.0)
    return z[:, 0]


def smoother_without_normalisation(weights, b):
    net = NO.fno_forward if isinstance(weights, dict) else NO.cnn_forward
    return net(weights, b)  # N(b) instead of N(b / ||b||) ||b||


def apply_without_alpha(H, l, x):
    if H.dim == 1:
        return _apply_level(H, l, x)
    M, K = H.ops[l]
    return K @ x @ K.T  # the alpha M X M^T term dropped


def apply_negated(H, l, x):
    return -_apply_level(H, l, x)  # b = y + A x*: residual sign flipped


def cholesky_solve_wrong_back_substitution(L, y):
    n = L.shape[0]
    z = np.array(y, dtype=np.float64, copy=True)
    for i in range(n):
        z[i] = (z[i] - L[i, :i] @ z[:i]) / L[i, i]
    x = z
    for i in range(n - 1, -1, -1):
        x[i] = (x[i] - L[i, i + 1:] @ x[i + 1:]) / L[i, i]  # row of L instead of column
    return x


def prolong_half_scale(H, l, e):
    Pm = _prolongation(H.size(l + 1)) / 2.0
    if H.dim == 1:
        return e @ Pm.T
    return Pm @ e @ Pm.T


def fno_drops_negative_rows(z, R):
    R2 = np.array(R, copy=True)
    R2[1] = 0.0  # the k1 in [n - m, n) block never applied
    return _fno_spectral(z, R2)


def fno_block0_for_both(z, R):
    R2 = np.array(R, copy=True)
    R2[1] = R2[0]  # block 0's weights reused for the k1 in [n - m, n) rows
    return _fno_spectral(z, R2)


def make_cycle(mistake):
    """The cycle of Algorithms 3/4 as the oracle runs it, with one step done
    wrongly: 'restrict_xstar' restricts y - A x* instead of y - A x (the
    smoothed iterate), 'filter_x' filters x* + h instead of h, 'smooth_y'
    smooths y instead of the defect b = y - A x*."""
    def cycle(H, weights, l, xstar, y, filt=True, trace=None):
        if l == H.levels - 1:
            B = y.shape[0]
            return NO.cholesky_solve(H.chol, y.reshape(B, -1).T).T.reshape(y.shape)
        xs = np.zeros_like(y) if xstar is None else xstar
        b = y - NO.apply_level(H, l, xs)
        h = NO.smoother(weights[l], y if mistake == "smooth_y" else b)
        if mistake == "filter_x":
            x = NO.spectral_filter(xs + h, H.dim) if filt else xs + h
        else:
            x = xs + (NO.spectral_filter(h, H.dim) if filt else h)
        xr = xs if mistake == "restrict_xstar" else x
        yc = NO.restrict(H, l, y - NO.apply_level(H, l, xr))
        return x + NO.prolong(H, l, NO.nmgf(H, weights, l + 1, None, yc, filt))
    return cycle


MUTANTS = {
    "cycle restricts the residual of x* instead of x": (
        "nmgf", make_cycle("restrict_xstar"),
        [P.test_linear_jacobi_smoother_reproduces_classical_backslash_mg]),
    "cycle filters x* + h instead of h": (
        "nmgf", make_cycle("filter_x"),
        [P.test_cycle_with_initial_guess_is_defect_correction]),
    "cycle smooths y instead of the defect": (
        "nmgf", make_cycle("smooth_y"),
        [P.test_cycle_with_initial_guess_is_defect_correction]),
    # (a Galerkin cycle with a zero smoother is invariant to the scale of R:
    # A_c = R A P and R y scale together, so only these pins can see it)
    "restriction without the 1/2": (
        "restriction", restriction_missing_half,
        [P.test_restriction_is_scaled_transpose_and_full_weighting,
         P.test_2d_transfer_is_kronecker,
         P.test_galerkin_2d_equals_dense_RAP]),
    "prolongation copies the last coarse value": (
        "prolongation", prolongation_copies_last_point,
        [P.test_prolongation_interpolates_linear_functions]),
    "filter symbol without the square root": (
        "filter_mask", mask_without_sqrt,
        [lambda: P.test_filter_1d_cosine_eigenvectors(16),
         P.test_filter_2d_cosine_products_and_special_vectors,
         P.test_filter_matches_bruteforce_dft]),
    "2D filter symbol with min instead of max": (
        "filter_mask", mask_min_instead_of_max,
        [P.test_filter_2d_cosine_products_and_special_vectors,
         P.test_filter_matches_bruteforce_dft]),
    "filter symbol on unshifted bins": (
        "filter_mask", mask_on_unshifted_bins,
        [lambda: P.test_filter_1d_cosine_eigenvectors(16),
         P.test_filter_matches_bruteforce_dft]),
    "convolution instead of cross-correlation": (
        "_conv_same", conv_flipped_kernel,
        [P.test_cnn_2d_matches_torch_conv, P.test_cnn_1d_matches_torch_conv]),
    "ReLU after the output layer": (
        "cnn_forward", cnn_relu_after_last_layer,
        [P.test_cnn_2d_matches_torch_conv]),
    "smoother without the norm scaling": (
        "smoother", smoother_without_normalisation,
        [P.test_smoother_is_positively_homogeneous_and_zero_safe,
         P.test_cycle_positive_homogeneity]),
    "operator apply without the alpha term": (
        "apply_level", apply_without_alpha,
        [lambda: P.test_2d_apply_matches_bruteforce_assembly(8, 1.0)]),
    "residual sign flipped": (
        "apply_level", apply_negated,
        [lambda: P.test_2d_apply_matches_bruteforce_assembly(8, 1.0),
         P.test_linear_jacobi_smoother_reproduces_classical_backslash_mg]),
    "back substitution with L instead of L^T": (
        "cholesky_solve", cholesky_solve_wrong_back_substitution,
        [P.test_coarse_cholesky_vs_scipy, P.test_single_level_cycle_is_exact_solve]),
    "prolongation of the correction at half scale": (
        "prolong", prolong_half_scale,
        [P.test_2d_transfer_is_kronecker,
         P.test_cycle_with_zero_smoother_is_pure_coarse_correction]),
    "FNO: negative-k1 block dropped": (
        "fno_spectral", fno_drops_negative_rows,
        [P.test_fno_spectral_identity_R_is_full_dft_projection,
         P.test_fno_spectral_blocks_act_on_their_own_rows]),
    "FNO: block 0 weights on both blocks": (
        "fno_spectral", fno_block0_for_both,
        [P.test_fno_spectral_blocks_act_on_their_own_rows]),
}


# problem data shared by the oracle and the CUDA path (nmg_inputs): mistakes
# there would pass every parity test, so their own pins must catch them
_aniso = I.aniso_regularisation_1d
_taps = I.gaussian_taps


def aniso_at_cell_centres(n, a=I.aniso_coefficient):
    return _aniso(n, a=lambda z: a(z + 0.5 / n))  # a at cell centres, not faces


def aniso_off_diagonal_sign(n, a=I.aniso_coefficient):
    diag, off = _aniso(n, a)
    return diag, -off


def taps_not_normalised(sigma):
    w = int(np.ceil(4.0 * sigma))
    j = np.arange(0, w + 1, dtype=np.float64)
    return np.exp(-(j * j) / (2.0 * sigma * sigma))


INPUT_MUTANTS = {
    "anisotropic coefficient at cell centres": (
        "aniso_regularisation_1d", aniso_at_cell_centres, [P.test_aniso_energy_identity]),
    "anisotropic off-diagonal sign": (
        "aniso_regularisation_1d", aniso_off_diagonal_sign,
        [P.test_aniso_constant_coefficient_is_dirichlet_laplacian, P.test_aniso_energy_identity]),
    "PSF taps not normalised": (
        "gaussian_taps", taps_not_normalised, [lambda: TI.test_gaussian_taps(2.0)]),
}


@pytest.mark.parametrize("mutant", sorted(INPUT_MUTANTS))
def test_input_pins_catch_planted_mistake(monkeypatch, mutant):
    name, fn, pins = INPUT_MUTANTS[mutant]
    monkeypatch.setattr(I, name, fn)
    for pin in pins:
        with pytest.raises(CAUGHT):
            pin()


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(monkeypatch, mutant):
    name, fn, pins = MUTANTS[mutant]
    _plant(monkeypatch, name, fn)
    for pin in pins:
        with pytest.raises(CAUGHT):
            pin()


def test_cycle_copy_without_mistake_passes_the_pins(monkeypatch):
    """Control for the cycle mutants: the same copy of the cycle with no
    mistake passes the pins they fail."""
    _plant(monkeypatch, "nmgf", make_cycle(None))
    P.test_linear_jacobi_smoother_reproduces_classical_backslash_mg()
    P.test_cycle_with_initial_guess_is_defect_correction()
    P.test_cycle_with_zero_smoother_is_pure_coarse_correction()
    P.test_cycle_positive_homogeneity()
