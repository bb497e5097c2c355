"""nmg_residual_noalloc, the residual step whose scratch is a fixed array
compiled into the library (no device allocation at call time), against
the allocating entry point nmg_residual on the same inputs.

Both run the same kernels on the same data, so they are expected to agree
bitwise; the bar is the single-step parity tolerance of the level type
(fp32 2e-5, fp64 1e-12, norm-wise relative).  Each case calls the new
entry point twice in a row (the array is shared between calls and nothing
in it is cleared in between).  The file is named to run last: it must pass
alone in a fresh process and after the rest of the suite.
"""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402

WDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2603_01064_gb300", "weights")
TOL = {"fp32": 2e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(ctx, G, level, x, y, r, B=None):
    """One call through the C ABI; returns (status, host norms)."""
    B = x.shape[0] if B is None else B
    norms = (ctypes.c_double * max(B, 1))()
    st = nmg.lib().nmg_residual_noalloc(ctx._h, G._h, level, B, _ptr(x), _ptr(y), _ptr(r), norms)
    return st, np.array(norms[:B])


def _rel(a, b):
    """Largest per-RHS max(norm-wise, element-wise) relative difference."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    nw = np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)
    ew = np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)
    return np.max(np.maximum(nw, ew))


def _check_twice(ctx, G, level, x, y, tol):
    r_ref = torch.empty_like(x)
    n_ref = G.residual(level, x, y, r_ref, norms=True)
    ref = r_ref.double().cpu().numpy()
    for _ in range(2):
        r = torch.full_like(x, float("nan"))
        st, nrm = _noalloc(ctx, G, level, x, y, r)
        assert st == 0, nmg.lib().nmg_last_error(ctx._h)
        assert _rel(r.double().cpu().numpy(), ref) <= tol
        assert np.max(np.abs(nrm - n_ref) / n_ref) <= tol


@pytest.mark.parametrize("prec,level", [("fp32", 0), ("fp32", 2), ("fp64", 0)])
def test_2d_matches_nmg_residual(ctx, prec, level):
    G = nmg.Hierarchy(ctx, dim=2, n=128, levels=5, alpha=1e-2, taps=I.gaussian_taps(2.0),
                      precision=prec, weights=I.random_cnn_weights(2, 4, seed=3))
    n = 128 >> level
    dt = torch.float32 if prec == "fp32" else torch.float64
    g = torch.Generator(device="cuda").manual_seed(11 + level)
    x = torch.randn((24, n, n), generator=g, device="cuda", dtype=dt)
    y = torch.randn((24, n, n), generator=g, device="cuda", dtype=dt)
    _check_twice(ctx, G, level, x, y, TOL[prec])
    G.close()


def _need(B, nt):
    r = lambda b: (b + 255) // 256 * 256  # noqa: E731
    return r(4 * B) + r(8 * nt * B) + r(8 * B)


def test_1d_largest_batch_and_limit(ctx):
    """1D n = 256 (32 residual tiles): the largest batch that fits the array
    matches nmg_residual twice; one more right-hand side is refused before
    any launch with NMG_ERR_ARG and a message giving the bytes."""
    col = I.kernel_column_1d(256)
    W = nmg.load_weights(os.path.join(WDIR, "c1_1d_n256_a1e-3.npz"))
    G = nmg.Hierarchy(ctx, dim=1, n=256, levels=3, alpha=1e-3, taps=col, precision="fp64",
                      weights=W)
    nt = (256 + 7) // 8
    bmax = max(b for b in range(1, 8192) if _need(b, nt) <= nmg.NOALLOC_SCRATCH_BYTES)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((bmax + 1, 256), generator=g, device="cuda", dtype=torch.float64)
    y = torch.randn((bmax + 1, 256), generator=g, device="cuda", dtype=torch.float64)
    _check_twice(ctx, G, 0, x[:bmax], y[:bmax], TOL["fp64"])
    r = torch.zeros_like(x)
    st, _ = _noalloc(ctx, G, 0, x, y, r)
    assert st == -1
    msg = nmg.lib().nmg_last_error(ctx._h).decode()
    assert "bytes" in msg and str(nmg.NOALLOC_SCRATCH_BYTES) in msg
    assert torch.count_nonzero(r).item() == 0  # nothing was launched
    G.close()


def test_binding_without_and_with_norms(ctx):
    """The binding's Hierarchy.residual_noalloc: without norms (no norm
    kernel, no wait for the stream: r is read after a synchronize) and with
    norms, twice each, against nmg_residual."""
    G = nmg.Hierarchy(ctx, dim=2, n=64, levels=4, alpha=1e-2, taps=I.gaussian_taps(2.0),
                      precision="fp32", weights=I.random_cnn_weights(2, 3, seed=6))
    g = torch.Generator(device="cuda").manual_seed(21)
    x = torch.randn((6, 64, 64), generator=g, device="cuda")
    y = torch.randn((6, 64, 64), generator=g, device="cuda")
    r_ref = torch.empty_like(x)
    n_ref = G.residual(0, x, y, r_ref, norms=True)
    ref = r_ref.double().cpu().numpy()
    for _ in range(2):
        r = torch.full_like(x, float("nan"))
        assert G.residual_noalloc(0, x, y, r, norms=False) is None
        torch.cuda.synchronize()
        assert _rel(r.double().cpu().numpy(), ref) <= TOL["fp32"]
    for _ in range(2):
        r = torch.full_like(x, float("nan"))
        nrm = G.residual_noalloc(0, x, y, r, norms=True)
        assert _rel(r.double().cpu().numpy(), ref) <= TOL["fp32"]
        assert np.max(np.abs(nrm - n_ref) / n_ref) <= TOL["fp32"]
    G.close()


def test_no_device_memory_taken(ctx):
    """After the set-up call, further calls leave the device's free memory
    unchanged.  The free-memory figure is device-wide: this assumes no other
    process allocates on the GPU meanwhile, so a difference is re-measured a
    few times before it counts."""
    G = nmg.Hierarchy(ctx, dim=2, n=64, levels=4, alpha=1e-2, taps=I.gaussian_taps(2.0),
                      precision="fp32", weights=I.random_cnn_weights(2, 3, seed=4))
    x = torch.randn((8, 64, 64), device="cuda")
    y = torch.randn((8, 64, 64), device="cuda")
    r = torch.empty_like(x)
    st, _ = _noalloc(ctx, G, 0, x, y, r)
    assert st == 0
    torch.cuda.synchronize()
    same = False
    for _attempt in range(3):
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            st, _ = _noalloc(ctx, G, 0, x, y, r)
            assert st == 0
        torch.cuda.synchronize()
        if torch.cuda.mem_get_info()[0] == free0:
            same = True
            break
    assert same
    G.close()
