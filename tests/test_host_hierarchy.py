"""The library's host-side set-up (no GPU): the Galerkin hierarchy that
nmg_setup builds from an operator description, read back through
nmg_host_level_dense and compared level by level with the FP64 oracle's
dense triple products (Algorithms 3/4: A_{l+1} = R A_l P; 2D through the 1D
factors, Section 4.2; the anisotropic 1D case of Section 4.1), plus the
argument checks the description goes through."""
import numpy as np
import pytest

import nmg_inputs as I
import oracle as O
import paper_2603_01064_gb300 as nmg


def close(a, b, rel=1e-14):
    return np.max(np.abs(a - b)) <= rel * np.max(np.abs(b))


@pytest.mark.parametrize("n,sigma,alpha,levels", [(32, 1.0, 1e-3, 3), (64, 2.0, 1e-2, 4),
                                                  (128, 4.0, 1e-1, 5)])
def test_2d_factors_match_oracle(n, sigma, alpha, levels):
    taps = I.gaussian_taps(sigma)
    H = O.build_hierarchy_2d(taps, n, alpha, levels)
    w = len(taps) - 1
    for l in range(levels):
        K, M = nmg.host_level_dense(dim=2, n=n, levels=levels, alpha=alpha, taps=taps, level=l)
        Mo, Ko = H.ops[l]
        assert K.shape == (n >> l, n >> l)
        assert close(K, Ko) and close(M, Mo), l
        # band half-width recursion w_{l+1} = floor(w_l / 2) + 1
        i, j = np.nonzero(K)
        assert np.max(np.abs(i - j)) <= w
        w = w // 2 + 1


def test_1d_operator_matches_oracle():
    n, alpha, levels = 256, 1e-3, 3
    col = I.kernel_column_1d(n)
    H = O.build_hierarchy_1d(col, alpha, levels)
    for l in range(levels):
        A = nmg.host_level_dense(dim=1, n=n, levels=levels, alpha=alpha, taps=col, level=l)
        assert close(A, H.ops[l]), l


def test_1d_anisotropic_operator_matches_oracle():
    n, alpha, levels = 256, 1e-5, 3
    col = I.kernel_column_1d(n)
    reg = I.aniso_regularisation_1d(n)
    H = O.build_hierarchy_1d(col, alpha, levels, reg=reg)
    for l in range(levels):
        A = nmg.host_level_dense(dim=1, n=n, levels=levels, alpha=alpha, taps=col, level=l,
                                 reg=reg)
        assert close(A, H.ops[l]), l


def test_description_errors():
    taps = I.gaussian_taps(2.0)
    ok = dict(dim=2, n=64, levels=4, alpha=1e-2, taps=taps)
    with pytest.raises(nmg.NMGError):  # level outside [0, levels)
        nmg.host_level_dense(**ok, level=4)
    with pytest.raises(nmg.NMGError):  # n not divisible by 2^(levels - 1)
        nmg.host_level_dense(**dict(ok, n=64, levels=8), level=0)
    with pytest.raises(nmg.NMGError):  # coarsest level above 1024 unknowns
        nmg.host_level_dense(**dict(ok, n=128, levels=2), level=0)
    with pytest.raises(nmg.NMGError):  # tridiagonal D is 1D only
        nmg.host_level_dense(**ok, level=0, reg=I.aniso_regularisation_1d(64))
    col = I.kernel_column_1d(64)
    with pytest.raises(nmg.NMGError):  # 1D needs the whole first column
        nmg.host_level_dense(dim=1, n=64, levels=2, alpha=1e-3, taps=col[:10], level=0)
