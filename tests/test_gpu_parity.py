"""GPU parity: every step and whole cycles of the CUDA path against the FP64
oracle on the same seeded inputs, through the C ABI.

Tolerances (norm-wise relative error unless stated):
  fp64: single steps 1e-12, one cycle 1e-10 (per-cycle iterate bound);
  fp32: single steps 2e-5, one cycle 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import oracle as O  # noqa: E402
from parity_err import rel_both  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402

TOL_STEP = {"fp64": 1e-12, "fp32": 2e-5}
TOL_CYCLE = {"fp64": 1e-10, "fp32": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32}


def relerr(a, b):
    """Largest per-RHS max(norm-wise, element-wise) relative error."""
    return np.max(rel_both(a, b))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


def dev(a, prec):
    return torch.tensor(np.ascontiguousarray(a), dtype=DT[prec], device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def make2d(ctx, prec, n=64, levels=4, sigma=2.0, alpha=1e-2, seed=3, filt=True):
    taps = I.gaussian_taps(sigma)
    W = I.random_cnn_weights(2, levels - 1, seed=seed)
    H = O.build_hierarchy_2d(taps, n, alpha, levels)
    G = nmg.Hierarchy(ctx, dim=2, n=n, levels=levels, alpha=alpha, taps=taps, precision=prec,
                      filter=filt, weights=W)
    return H, G, W


def make1d(ctx, n=256, levels=3, alpha=1e-3, seed=4, weights=None, filt=True):
    col = I.kernel_column_1d(n)
    W = weights if weights is not None else I.random_cnn_weights(1, levels - 1, seed=seed)
    H = O.build_hierarchy_1d(col, alpha, levels)
    G = nmg.Hierarchy(ctx, dim=1, n=n, levels=levels, alpha=alpha, taps=col, precision="fp64",
                      filter=filt, weights=W)
    return H, G, W


# ---------------------------------------------------------------------------
# setup (a1): the library's Galerkin factors equal the oracle's dense RAP
# ---------------------------------------------------------------------------

def test_hierarchy_factors_match_oracle(ctx):
    H, G, _ = make2d(ctx, "fp64", n=128, levels=5)
    for l in range(5):
        K, M = G.level_dense(l)
        Mo, Ko = H.ops[l]
        assert np.max(np.abs(K - Ko)) < 1e-15
        assert np.max(np.abs(M - Mo)) < 1e-15
    H1, G1, _ = make1d(ctx)
    for l in range(3):
        assert np.max(np.abs(G1.level_dense(l) - H1.ops[l])) < 1e-15


# ---------------------------------------------------------------------------
# single steps (2D)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_residual_and_norms(ctx, prec):
    H, G, _ = make2d(ctx, prec)
    rng = np.random.default_rng(1)
    for l in range(H.levels):
        m = H.size(l)
        x = rng.standard_normal((3, m, m))
        y = rng.standard_normal((3, m, m))
        xd, yd = dev(x, prec), dev(y, prec)
        rd = torch.empty_like(xd)
        norms = G.residual(l, xd, yd, rd, norms=True)
        ref = y - O.apply_level(H, l, x)
        assert relerr(host(rd), ref) < TOL_STEP[prec]
        assert np.max(np.abs(norms - np.linalg.norm(ref.reshape(3, -1), axis=1)) /
                      np.linalg.norm(ref.reshape(3, -1), axis=1)) < TOL_STEP[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_residual_restrict(ctx, prec):
    H, G, _ = make2d(ctx, prec)
    rng = np.random.default_rng(2)
    for l in range(H.levels - 1):
        m = H.size(l)
        x = rng.standard_normal((2, m, m))
        y = rng.standard_normal((2, m, m))
        yc = torch.empty((2, m // 2, m // 2), dtype=DT[prec], device="cuda")
        G.residual_restrict(l, dev(x, prec), dev(y, prec), yc)
        ref = O.restrict(H, l, y - O.apply_level(H, l, x))
        assert relerr(host(yc), ref) < TOL_STEP[prec]


@pytest.mark.parametrize("sigma,n", [(4.0, 256), (8.0, 256), (4.0, 512)])
def test_wide_stencil_residual_and_restrict(ctx, sigma, n):
    """fp32 fine level with a wide PSF stencil (half-width 16 or 32): the
    strip residual r = y - A x with its norms, and the residual followed by
    the separate full-weighting restriction, against the oracle's dense
    factors; x, y with a zero right-hand side inside the batch."""
    taps = I.gaussian_taps(sigma)
    L = int(np.log2(n // 32)) + 1  # coarsest level 32 x 32
    H = O.build_hierarchy_2d(taps, n, 1e-2, L)
    G = nmg.Hierarchy(ctx, dim=2, n=n, levels=L, alpha=1e-2, taps=taps, precision="fp32",
                      weights=I.random_cnn_weights(2, L - 1, seed=8))
    rng = np.random.default_rng(int(sigma) + n)
    x = rng.standard_normal((3, n, n))
    y = rng.standard_normal((3, n, n))
    x[1] = 0.0
    y[1] = 0.0
    xd, yd = dev(x, "fp32"), dev(y, "fp32")
    x32, y32 = host(xd), host(yd)
    rd = torch.empty_like(xd)
    norms = G.residual(0, xd, yd, rd, norms=True)
    ref = y32 - O.apply_level(H, 0, x32)
    keep = [0, 2]
    got = host(rd)
    assert np.all(got[1] == 0.0) and norms[1] == 0.0
    assert relerr(got[keep], ref[keep]) < TOL_STEP["fp32"]
    nref = np.linalg.norm(ref.reshape(3, -1), axis=1)[keep]
    assert np.max(np.abs(norms[keep] - nref) / nref) < TOL_STEP["fp32"]
    yc = torch.full((3, n // 2, n // 2), 7.0, dtype=torch.float32, device="cuda")
    G.residual_restrict(0, xd, yd, yc)
    refc = O.restrict(H, 0, ref)
    gotc = host(yc)
    assert np.all(gotc[1] == 0.0)
    assert relerr(gotc[keep], refc[keep]) < TOL_STEP["fp32"]
    G.close()


@pytest.mark.parametrize("kch", [1, 3, 5, 16])
def test_wide_stencil_chunk_counts(ctx, tmp_path, kch):
    """The wide strip kernels cut every 64-column strip into kch chunks
    (512 rows: 3 and 5 leave a shorter last chunk), dealt block-cyclically
    over the SMs: residual with norms and residual + restriction at each
    chunk count, forced through the tuner's cache, against the oracle."""
    from tuning_util import force_tuning
    n, sigma, L = 512, 4.0, 5
    taps = I.gaussian_taps(sigma)
    H = O.build_hierarchy_2d(taps, n, 1e-2, L)
    G = nmg.Hierarchy(ctx, dim=2, n=n, levels=L, alpha=1e-2, taps=taps, precision="fp32",
                      weights=I.random_cnn_weights(2, L - 1, seed=9))
    force_tuning(G, 3, tmp_path / "tune.txt", {0: dict(res=-kch, rst=-kch)})
    t = G.tuning(0)
    assert t["res_tile"] == -kch and t["rst_tile"] == -kch
    rng = np.random.default_rng(kch)
    x = rng.standard_normal((3, n, n))
    y = rng.standard_normal((3, n, n))
    xd, yd = dev(x, "fp32"), dev(y, "fp32")
    x32, y32 = host(xd), host(yd)
    rd = torch.empty_like(xd)
    norms = G.residual(0, xd, yd, rd, norms=True)
    ref = y32 - O.apply_level(H, 0, x32)
    assert relerr(host(rd), ref) < TOL_STEP["fp32"]
    nref = np.linalg.norm(ref.reshape(3, -1), axis=1)
    assert np.max(np.abs(norms - nref) / nref) < TOL_STEP["fp32"]
    yc = torch.full((3, n // 2, n // 2), 7.0, dtype=torch.float32, device="cuda")
    G.residual_restrict(0, xd, yd, yc)
    assert relerr(host(yc), O.restrict(H, 0, ref)) < TOL_STEP["fp32"]
    G.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_smoother(ctx, prec):
    H, G, W = make2d(ctx, prec)
    rng = np.random.default_rng(3)
    for l in range(H.levels - 1):
        m = H.size(l)
        b = rng.standard_normal((3, m, m)) * np.array([1.0, 1e-3, 50.0])[:, None, None]
        hd = torch.empty((3, m, m), dtype=DT[prec], device="cuda")
        G.smooth(l, dev(b, prec), hd)
        ref = O.smoother(W[l], b)
        assert relerr(host(hd), ref) < 10 * TOL_STEP[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_smoother_zero_input(ctx, prec):
    H, G, W = make2d(ctx, prec)
    b = torch.zeros((2, 64, 64), dtype=DT[prec], device="cuda")
    hd = torch.full((2, 64, 64), 7.0, dtype=DT[prec], device="cuda")
    G.smooth(0, b, hd)
    assert torch.count_nonzero(hd).item() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_filter_update(ctx, prec):
    H, G, _ = make2d(ctx, prec)
    rng = np.random.default_rng(4)
    for l in range(H.levels - 1):
        m = H.size(l)
        h = rng.standard_normal((2, m, m))
        xs = rng.standard_normal((2, m, m))
        xd = dev(xs, prec)
        G.filter_update(l, xd, dev(h, prec), xd)  # in place: x = x* + F'(h)
        ref = xs + O.spectral_filter(h, 2)
        assert relerr(host(xd), ref) < TOL_STEP[prec]
        out = torch.empty_like(xd)
        G.filter_update(l, None, dev(h, prec), out)
        assert relerr(host(out), O.spectral_filter(h, 2)) < TOL_STEP[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [256, 512])
def test_filter_update_large_levels(ctx, prec, n):
    """The warp-level three-pass filter of 256 x 256 and 512 x 512 levels
    (row pairs, column pairs through shared memory, rows), in place and from
    a zero x*, with a zero image in the batch (its F'(h) is 0)."""
    taps = I.gaussian_taps(2.0)
    L = int(np.log2(n // 32)) + 1  # coarsest level 32 x 32
    G = nmg.Hierarchy(ctx, dim=2, n=n, levels=L, alpha=1e-2, taps=taps, precision=prec,
                      weights=I.random_cnn_weights(2, L - 1, seed=7))
    rng = np.random.default_rng(n)
    h = rng.standard_normal((3, n, n))
    h[1] = 0.0
    xs = rng.standard_normal((3, n, n))
    xd = dev(xs, prec)
    G.filter_update(0, xd, dev(h, prec), xd)
    ref = xs + O.spectral_filter(h, 2)
    assert relerr(host(xd), ref) < TOL_STEP[prec]
    out = torch.empty_like(xd)
    G.filter_update(0, None, dev(h, prec), out)
    got = host(out)
    assert np.all(got[1] == 0.0)
    keep = [0, 2]
    assert relerr(got[keep], O.spectral_filter(h[keep], 2)) < TOL_STEP[prec]
    G.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_coarse_and_prolong(ctx, prec):
    H, G, _ = make2d(ctx, prec)
    rng = np.random.default_rng(5)
    nc = H.size(H.levels - 1)
    y = rng.standard_normal((3, nc, nc))
    xd = torch.empty((3, nc, nc), dtype=DT[prec], device="cuda")
    G.coarse_solve(dev(y, prec), xd)
    ref = O.cholesky_solve(H.chol, y.reshape(3, -1).T).T.reshape(3, nc, nc)
    assert relerr(host(xd), ref) < 10 * TOL_STEP[prec]
    for l in range(H.levels - 1):
        m = H.size(l)
        e = rng.standard_normal((2, m // 2, m // 2))
        x = rng.standard_normal((2, m, m))
        xd = dev(x, prec)
        G.prolong_correct(l, dev(e, prec), xd)
        assert relerr(host(xd), x + O.prolong(H, l, e)) < TOL_STEP[prec]


# ---------------------------------------------------------------------------
# one cycle from the same state (per-cycle iterate parity)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("filt", [True, False])
def test_one_cycle_2d(ctx, prec, filt):
    H, G, W = make2d(ctx, prec, filt=filt)
    rng = np.random.default_rng(6)
    f = rng.standard_normal((4, 64, 64))
    u0 = rng.standard_normal((4, 64, 64)) * 0.1
    u0[0] = 0.0  # the paper's x^0 = 0
    ud = dev(u0, prec)
    G.cycle(dev(f, prec), ud)
    ref = O.nmgf(H, W, 0, u0, f, filt=filt)
    assert relerr(host(ud), ref) < TOL_CYCLE[prec]


def test_one_cycle_ragged_small_levels(ctx):
    """n = 64 with 5 levels: smoother on an 8x8 grid (smaller than a tile) and a
    4x4 coarsest grid."""
    H, G, W = make2d(ctx, "fp64", n=64, levels=5, sigma=1.0)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((3, 64, 64))
    ud = torch.zeros((3, 64, 64), dtype=torch.float64, device="cuda")
    G.cycle(dev(f, "fp64"), ud)
    ref = O.nmgf(H, W, 0, None, f)
    assert relerr(host(ud), ref) < TOL_CYCLE["fp64"]


def test_one_cycle_single_level_is_exact(ctx):
    taps = I.gaussian_taps(1.0)
    G = nmg.Hierarchy(ctx, dim=2, n=8, levels=1, alpha=1e-2, taps=taps, precision="fp64")
    H = O.build_hierarchy_2d(taps, 8, 1e-2, 1)
    f = np.random.default_rng(8).standard_normal((2, 8, 8))
    ud = torch.zeros((2, 8, 8), dtype=torch.float64, device="cuda")
    G.cycle(dev(f, "fp64"), ud)
    assert relerr(host(ud), O.nmgf(H, [], 0, None, f)) < 1e-12


# ---------------------------------------------------------------------------
# 1D (Algorithm 3), fp64
# ---------------------------------------------------------------------------

def test_1d_steps(ctx):
    H, G, W = make1d(ctx)
    rng = np.random.default_rng(9)
    for l in range(2):
        m = H.size(l)
        x, y = rng.standard_normal((2, m)), rng.standard_normal((2, m))
        rd = torch.empty((2, m), dtype=torch.float64, device="cuda")
        G.residual(l, dev(x, "fp64"), dev(y, "fp64"), rd)
        assert relerr(host(rd), y - O.apply_level(H, l, x)) < 1e-13
        yc = torch.empty((2, m // 2), dtype=torch.float64, device="cuda")
        G.residual_restrict(l, dev(x, "fp64"), dev(y, "fp64"), yc)
        assert relerr(host(yc), O.restrict(H, l, y - O.apply_level(H, l, x))) < 1e-13
        hd = torch.empty((2, m), dtype=torch.float64, device="cuda")
        G.smooth(l, dev(y, "fp64"), hd)
        assert relerr(host(hd), O.smoother(W[l], y)) < 1e-12
        xd = dev(x, "fp64")
        G.filter_update(l, xd, dev(y, "fp64"), xd)
        assert relerr(host(xd), x + O.spectral_filter(y, 1)) < 1e-12


def test_1d_one_cycle(ctx):
    H, G, W = make1d(ctx)
    rng = np.random.default_rng(10)
    f = rng.standard_normal((5, 256))
    u0 = 0.01 * rng.standard_normal((5, 256))
    ud = dev(u0, "fp64")
    G.cycle(dev(f, "fp64"), ud)
    assert relerr(host(ud), O.nmgf(H, W, 0, u0, f)) < TOL_CYCLE["fp64"]


# ---------------------------------------------------------------------------
# argument checking (no launch happens for any of these)
# ---------------------------------------------------------------------------

def test_setup_argument_errors(ctx):
    taps = I.gaussian_taps(2.0)
    with pytest.raises(nmg.NMGError) as e:
        nmg.Hierarchy(ctx, dim=2, n=96, levels=4, alpha=1e-2, taps=taps, precision="fp32",
                      weights=I.random_cnn_weights(2, 3, 0))
    assert e.value.code == -1
    with pytest.raises(nmg.NMGError) as e:
        nmg.Hierarchy(ctx, dim=2, n=64, levels=4, alpha=1e-2, taps=taps, precision="fp32",
                      weights=I.random_cnn_weights(2, 2, 0))
    assert e.value.code == -6
    with pytest.raises(nmg.NMGError) as e:
        nmg.Hierarchy(ctx, dim=2, n=64, levels=4, alpha=-1.0, taps=taps, precision="fp32",
                      weights=I.random_cnn_weights(2, 3, 0))
    assert e.value.code == -3


def test_batch_zero_is_noop(ctx):
    H, G, W = make2d(ctx, "fp32")
    f = torch.zeros((0, 64, 64), dtype=torch.float32, device="cuda")
    cyc, st, rr = G.solve(f, f.clone())
    assert len(cyc) == 0


@pytest.mark.parametrize("prec", ["fp32", "bf16_refine"])
def test_host_buffer_solves_match_device_solve(ctx, prec):
    """nmg_solve_host (f and u copied in, u copied back) and
    nmg_solve_host_zero (zero initial guess; u is output only, here filled
    with NaN beforehand) give bitwise the same iterate and per-RHS
    information as nmg_solve on device buffers."""
    H, G, W = make2d(ctx, prec)
    f, _ = I.rhs_2d_ellipses_grf(64, 3, seed=77, sigma=2.0)
    udt = np.float32 if prec == "fp32" else np.float64
    fd = dev(f, "fp32")
    ud = torch.zeros((3, 64, 64), dtype=torch.float32 if prec == "fp32" else torch.float64,
                     device="cuda")
    ref = G.solve(fd, ud, rtol=1e-12, max_cycles=4)
    u_dev = host(ud)
    fh = np.ascontiguousarray(f, dtype=np.float32)
    u1 = np.zeros((3, 64, 64), dtype=udt)
    got1 = G.solve_host(fh, u1, rtol=1e-12, max_cycles=4)
    u2 = np.full((3, 64, 64), np.nan, dtype=udt)
    got2 = G.solve_host(fh, u2, rtol=1e-12, max_cycles=4, zero_start=True)
    for got, u in ((got1, u1), (got2, u2)):
        for a, b in zip(got, ref):
            assert np.array_equal(np.asarray(a), np.asarray(b))
        assert np.array_equal(u.astype(np.float64), u_dev)
