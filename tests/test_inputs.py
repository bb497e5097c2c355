"""The seeded input generators follow the stated recipe: normalised PSF taps
truncated at 4 sigma, blurs that are the operator's own K (zero boundary),
1 % relative noise, and right-hand sides that depend only on their seed."""
import numpy as np
import pytest

import nmg_inputs as I
import oracle as O


@pytest.mark.parametrize("sigma", [1.0, 2.0, 4.0, 8.0])
def test_gaussian_taps(sigma):
    g = I.gaussian_taps(sigma)
    assert len(g) == int(np.ceil(4 * sigma)) + 1
    assert abs(g[0] + 2 * g[1:].sum() - 1.0) < 1e-15
    assert np.all(np.diff(g) < 0)
    assert abs(g[1] / g[0] - np.exp(-1 / (2 * sigma ** 2))) < 1e-14


def test_blurs_are_the_operators_K():
    rng = np.random.default_rng(0)
    taps = I.gaussian_taps(2.0)
    u = rng.standard_normal((2, 24, 24))
    K = O.banded_toeplitz(taps, 24)
    assert np.max(np.abs(I.blur_2d(u, taps) - K @ u @ K.T)) < 1e-14
    col = I.kernel_column_1d(64)
    v = rng.standard_normal((3, 64))
    assert np.max(np.abs(I.blur_1d(v, col) - v @ O.toeplitz_from_column(col).T)) < 1e-14


@pytest.mark.parametrize("gen,args", [
    (I.rhs_1d_sines_steps, (256, 64, 11)),
    (I.rhs_2d_ellipses_grf, (64, 16, 12, 2.0)),
    (I.rhs_2d_waves_rects, (64, 16, 13, 2.0)),
])
def test_rhs_noise_level_and_seeding(gen, args):
    f, u = gen(*args)
    f2, u2 = gen(*args)
    assert np.array_equal(f, f2) and np.array_equal(u, u2)
    f3, _ = gen(*args[:2], args[2] + 1, *args[3:])
    assert not np.array_equal(f, f3)
    if f.ndim == 2:
        clean = I.blur_1d(u, I.kernel_column_1d(f.shape[1]))
    else:
        clean = I.blur_2d(u, I.gaussian_taps(args[3]))
    axes = tuple(range(1, f.ndim))
    ratio = np.sqrt(np.mean((f - clean) ** 2, axis=axes) / np.mean(clean ** 2, axis=axes))
    m = np.prod(f.shape[1:])
    assert np.all(np.abs(ratio - 0.01) < 0.01 * 5 / np.sqrt(m))  # 1 % noise, 5 std errors
