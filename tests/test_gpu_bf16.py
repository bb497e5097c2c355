"""GPU parity of the bf16 refinement forms (tensor-core smoother, compensated
fp32 outer residual, fp64 update) against the FP64 oracle.

* bf16_refine (every operand three bf16 terms, six products): the smoother
  against the un-rounded FP64 oracle at 1e-5 (fp32-level operands and fp32
  accumulation), one refinement step and the first trained cycles at 1e-4
  (the per-cycle bar of the bf16 form is 1e-3).
* bf16x3_refine (operand pairs hi + lo, three products): the smoother at
  1e-4, one refinement step and trained cycles at 1e-3.
* fp16_refine (split operands in fp16, power-of-two-scaled network): the
  smoother against FP64 at 1e-5 (hi + lo fp16 carries 2^-22 relative; the
  scaling is exact), one refinement step and the first trained cycles at
  1e-4.
* bf16fast_refine (one bf16 per operand): compared with a CPU evaluation of
  the same network that rounds to bf16 exactly where the kernels store bf16
  (hidden activations, hidden-layer weights) and accumulates in fp64: the
  two may differ only by fp32 accumulation order, which pins the MMA
  operand layout (1e-3: accumulation order can flip a few bf16 roundings);
  its solve must still reach the tolerance.
* Full solves reach ||f - A u|| / ||f|| <= 1e-6 as measured by the oracle's
  own fp64 apply.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import oracle as O  # noqa: E402
from parity_err import rel_both  # noqa: E402
from oracle import nmg_oracle as ON  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402

WDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2603_01064_gb300", "weights")
C2W = os.path.join(WDIR, "c2_2d_n128_s2_a1e-2.npz")


def bf16(a):
    """Round to bf16 (round to nearest even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def emulated_fast(W, b):
    """s N(b/s) rounded to bf16 exactly where the fast kernels store bf16: the
    activations that feed a hidden layer and the hidden layers' weights (the
    first and the output layer run in fp32; the last hidden layer's
    activations go to the fused output layer in fp32)."""
    s = np.sqrt(np.sum(b.reshape(b.shape[0], -1) ** 2, axis=1))[:, None, None]
    x = (b / s)[:, None]
    last = len(W) - 1
    for i, (w, bias) in enumerate(W):
        wi = np.asarray(w, np.float32).astype(np.float64) if i in (0, last) else bf16(w)
        x = ON._conv_same(x, wi, np.asarray(bias, np.float32).astype(np.float64))
        x = x.astype(np.float32).astype(np.float64)  # the kernels accumulate in fp32
        if i < last:
            x = np.maximum(x, 0.0)
            if i < last - 1:
                x = bf16(x)
    return x[:, 0] * s


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


def make(ctx, prec="bf16_refine", n=64, levels=4, sigma=2.0, alpha=1e-2, seed=21, weights=None):
    taps = I.gaussian_taps(sigma)
    W = weights if weights is not None else I.random_cnn_weights(2, levels - 1, seed=seed)
    G = nmg.Hierarchy(ctx, dim=2, n=n, levels=levels, alpha=alpha, taps=taps, precision=prec,
                      weights=W)
    H = O.build_hierarchy_2d(taps, n, alpha, levels)
    return H, G, W


def rel(a, b):
    """Largest per-RHS max(norm-wise, element-wise) relative error."""
    return np.max(rel_both(a, b))


def smooth_gpu(G, l, b):
    bd = torch.tensor(b, dtype=torch.float32, device="cuda")
    hd = torch.full_like(bd, 5.0)
    G.smooth(l, bd, hd)
    torch.cuda.synchronize()
    return bd.double().cpu().numpy(), hd.double().cpu().numpy()


def test_fast_smoother_matches_bf16_emulation(ctx):
    H, G, W = make(ctx, "bf16fast_refine")
    rng = np.random.default_rng(1)
    for l in range(H.levels - 1):
        m = H.size(l)
        b = rng.standard_normal((3, m, m)) * np.array([1.0, 1e-4, 30.0])[:, None, None]
        b32, h = smooth_gpu(G, l, b)
        # fp32 accumulation order can flip a few bf16 roundings of hidden
        # activations (2^-8 each); an operand-layout error would be O(1)
        assert rel(h, emulated_fast(W[l], b32)) < 1e-3, l


SPLIT_TOL = {"bf16_refine": 1e-5, "bf16x3_refine": 1e-4, "fp16_refine": 1e-5}


@pytest.mark.parametrize("prec", ["bf16_refine", "bf16x3_refine", "bf16fast_refine", "fp16_refine"])
def test_smoother_small_level_and_zero_rhs(ctx, prec):
    """An 8x8 level (smaller than the 16x16 tile) and a zero right-hand side."""
    H, G, W = make(ctx, prec, n=64, levels=5, sigma=1.0)
    b = np.random.default_rng(2).standard_normal((2, 8, 8))
    b[1] = 0.0
    b32, h = smooth_gpu(G, 3, b)
    assert np.all(h[1] == 0.0)
    if prec == "bf16fast_refine":
        assert rel(h[:1], emulated_fast(W[3], b32[:1])) < 1e-3
    else:
        assert rel(h[:1], O.smoother(W[3], b32[:1])) < SPLIT_TOL[prec]


@pytest.mark.parametrize("prec", ["bf16_refine", "bf16x3_refine", "fp16_refine", "bf16top_refine"])
def test_split_smoother_matches_fp64(ctx, prec):
    H, G, W = make(ctx, prec)
    rng = np.random.default_rng(3)
    for l in range(H.levels - 1):
        m = H.size(l)
        b = rng.standard_normal((3, m, m)) * np.array([1.0, 1e-4, 30.0])[:, None, None]
        b32, h = smooth_gpu(G, l, b)
        tol = SPLIT_TOL[prec] if prec != "bf16top_refine" else \
            SPLIT_TOL["bf16_refine" if l == 0 else "bf16x3_refine"]
        assert rel(h, O.smoother(W[l], b32)) < tol, l


@pytest.mark.parametrize("prec", ["bf16_refine", "bf16x3_refine", "fp16_refine"])
@pytest.mark.parametrize("layers", [3, 4, 5])
def test_split_smoother_depths_and_zero_rhs(ctx, prec, layers):
    """On levels of side >= 32 the split forms compute the first layer inside
    the first hidden layer's kernel when another hidden layer follows (4 and
    5 layers; 3 layers keep the separate first-layer kernel).  A zero
    right-hand side between nonzero ones is skipped by the tile schedule
    and gets h = 0; the others match the FP64 oracle."""
    W = I.random_cnn_weights(2, 2, seed=40 + layers, layers=layers)
    H, G, W = make(ctx, prec, n=64, levels=3, weights=W)
    rng = np.random.default_rng(layers)
    for l in range(2):
        m = H.size(l)
        b = rng.standard_normal((4, m, m)) * np.array([1.0, 1.0, 1e-3, 20.0])[:, None, None]
        b[1] = 0.0
        b32, h = smooth_gpu(G, l, b)
        assert np.all(h[1] == 0.0)
        keep = [0, 2, 3]
        assert rel(h[keep], O.smoother(W[l], b32[keep])) < SPLIT_TOL[prec], (l, layers)


def _mixed_depth_weights(depths, seed):
    """Seeded random CNN weights with a different depth on every level."""
    return [I.random_cnn_weights(2, 1, seed=seed + l, layers=d)[0] for l, d in enumerate(depths)]


@pytest.mark.parametrize("prec", ["bf16_refine", "fp16_refine", "fp32", "fp64"])
def test_per_level_depths(ctx, prec):
    """Smoother levels of different depth (4, 12, 3 layers; the deep one is
    the receptive field a transition level needs, Appendix A sizes every
    level's net separately): each level's smoother and one whole cycle
    against the FP64 oracle with the same weights."""
    W = _mixed_depth_weights([4, 12, 3], seed=70)
    H, G, W = make(ctx, prec, n=64, levels=4, weights=W)
    rng = np.random.default_rng(71)
    tol = {"fp64": 1e-12, "fp32": 2e-5}.get(prec, SPLIT_TOL.get(prec))
    for l in range(3):
        m = H.size(l)
        b = rng.standard_normal((3, m, m)) * np.array([1.0, 1e-3, 20.0])[:, None, None]
        if prec == "fp64":
            bd = torch.tensor(b, dtype=torch.float64, device="cuda")
            hd = torch.zeros_like(bd)
            G.smooth(l, bd, hd)
            torch.cuda.synchronize()
            assert rel(hd.cpu().numpy(), O.smoother(W[l], b)) < tol, l
        else:
            b32, h = smooth_gpu(G, l, b)
            assert rel(h, O.smoother(W[l], b32)) < tol, (l, prec)
    f = rng.standard_normal((3, 64, 64))
    dt = torch.float64 if prec == "fp64" else torch.float32
    fd = torch.tensor(f, dtype=dt, device="cuda")
    f_in = fd.double().cpu().numpy()
    udt = torch.float64 if prec in ("fp64", "bf16_refine", "fp16_refine") else torch.float32
    ud = torch.zeros(fd.shape, dtype=udt, device="cuda")
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    ctol = {"fp64": 1e-10, "fp32": 1e-5}.get(prec, CYCLE_TOL.get(prec))
    assert rel(ud.double().cpu().numpy(), O.nmgf(H, W, 0, None, f_in)) < ctol


def test_per_level_depth_limits(ctx):
    """More than 16 layers on a level, or fewer than 3 in a tensor-core
    form, is refused at setup with a status, not at the first launch."""
    with pytest.raises(nmg.NMGError) as e:
        make(ctx, "fp32", n=64, levels=3, weights=_mixed_depth_weights([4, 17], seed=80))
    assert e.value.code == -7  # NMG_ERR_UNSUPPORTED
    with pytest.raises(nmg.NMGError):
        make(ctx, "bf16_refine", n=64, levels=3, weights=_mixed_depth_weights([4, 2], seed=81))
    make(ctx, "fp32", n=64, levels=3, weights=_mixed_depth_weights([4, 2], seed=81))


CYCLE_TOL = {"bf16_refine": 1e-4, "bf16x3_refine": 1e-3, "fp16_refine": 1e-4,
             "bf16top_refine": 1e-3}


@pytest.mark.parametrize("prec", ["bf16_refine", "bf16x3_refine", "fp16_refine", "bf16top_refine"])
def test_refine_step_matches_fp64_cycle(ctx, prec):
    H, G, W = make(ctx, prec)
    rng = np.random.default_rng(4)
    f = rng.standard_normal((4, 64, 64))
    u0 = 0.05 * rng.standard_normal((4, 64, 64))
    u0[0] = 0.0
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    f32 = fd.double().cpu().numpy()  # the fp32 right-hand side both sides see
    ud = torch.tensor(u0, dtype=torch.float64, device="cuda")
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    assert rel(ud.cpu().numpy(), O.nmgf(H, W, 0, u0, f32)) < CYCLE_TOL[prec]


@pytest.mark.parametrize("sigma", [4.0, 8.0])
def test_refine_step_wide_stencils(ctx, sigma):
    """The compensated outer residual's wide strip kernel (PSF half-width 16
    for sigma 4 px, 32 for sigma 8 px) inside one refinement step from a
    nonzero state on a 256 x 256 grid: the step's increment against the
    oracle cycle's from the same state."""
    n, L = 256, 4
    H, G, W = make(ctx, "bf16_refine", n=n, levels=L, sigma=sigma, alpha=1e-2, seed=31)
    rng = np.random.default_rng(int(sigma))
    f = rng.standard_normal((3, n, n))
    u0 = 0.2 * rng.standard_normal((3, n, n))
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    f32 = fd.double().cpu().numpy()
    ud = torch.tensor(u0, dtype=torch.float64, device="cuda")
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    ref = O.nmgf(H, W, 0, u0, f32)
    assert rel(ud.cpu().numpy() - u0, ref - u0) < 1e-4


@pytest.mark.parametrize("kch", [1, 3, 5, 16])
def test_refine_wide_chunk_counts(ctx, tmp_path, kch):
    """The compensated outer residual's wide strip kernel with kch chunks
    per strip (forced through the tuner's cache; 3 and 5 leave a shorter
    last chunk) inside one refinement step on a 512 x 512 grid (PSF
    half-width 16): the step's increment against the oracle cycle's."""
    from tuning_util import force_tuning
    n, L = 512, 5
    H, G, W = make(ctx, "bf16_refine", n=n, levels=L, sigma=4.0, alpha=1e-2, seed=33)
    force_tuning(G, 2, tmp_path / "tune.txt", {0: dict(ref=-kch)})
    assert G.tuning(0)["ref_tile"] == -kch
    rng = np.random.default_rng(40 + kch)
    f = rng.standard_normal((2, n, n))
    u0 = 0.2 * rng.standard_normal((2, n, n))
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    f32 = fd.double().cpu().numpy()
    ud = torch.tensor(u0, dtype=torch.float64, device="cuda")
    G.cycle(fd, ud)
    torch.cuda.synchronize()
    ref = O.nmgf(H, W, 0, u0, f32)
    assert rel(ud.cpu().numpy() - u0, ref - u0) < 1e-4


@pytest.fixture(scope="module")
def c2w():
    if not os.path.exists(C2W):
        pytest.skip("trained weights missing")
    return nmg.load_weights(C2W)


@pytest.mark.parametrize("prec", ["bf16_refine", "bf16x3_refine", "fp16_refine", "bf16top_refine"])
def test_trained_first_cycles_match_fp64(ctx, c2w, prec):
    """Per-cycle iterate parity with trained smoothers on the 128x128 operator:
    cycles 1..4 from the GPU's own previous iterate, each against one oracle
    cycle from the same state."""
    H, G, _ = make(ctx, prec, n=128, levels=5, weights=c2w)
    f, _ = I.rhs_2d_ellipses_grf(128, 3, seed=5, sigma=2.0)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    f32 = fd.double().cpu().numpy()
    ud = torch.zeros((3, 128, 128), dtype=torch.float64, device="cuda")
    for _ in range(4):
        up = ud.cpu().numpy().copy()
        G.cycle(fd, ud)
        torch.cuda.synchronize()
        assert rel(ud.cpu().numpy(), O.nmgf(H, c2w, 0, up, f32)) < CYCLE_TOL[prec]


@pytest.mark.parametrize("prec", ["bf16_refine", "bf16x3_refine", "bf16fast_refine", "fp16_refine"])
def test_refine_solve_trained_c2_reaches_tolerance(ctx, c2w, prec):
    H, G, _ = make(ctx, prec, n=128, levels=5, sigma=2.0, alpha=1e-2, weights=c2w)
    f, _ = I.rhs_2d_ellipses_grf(128, 8, seed=77, sigma=2.0)
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    ud = torch.zeros((8, 128, 128), dtype=torch.float64, device="cuda")
    cyc, st, rr = G.solve(fd, ud, rtol=1e-6, max_cycles=60)
    assert np.all(st == 0), (cyc, rr)
    f32 = fd.double().cpu().numpy()
    rr_oracle = O.relres(H, f32, ud.cpu().numpy())
    assert np.all(rr_oracle <= 1.01e-6), rr_oracle
    assert np.max(np.abs(rr_oracle - rr) / rr_oracle) < 1e-3
