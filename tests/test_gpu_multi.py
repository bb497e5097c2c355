"""Mixed-size batched solve (nmg_solve_multi): batches on hierarchies of
different grid sizes, operators and precisions solved in one outer loop
(one CUDA graph per iteration, items as parallel branches) give exactly the
results each batch gets when solved alone."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import nmg_inputs as I  # noqa: E402
import oracle as O  # noqa: E402
from parity_err import rel_both  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402

WDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2603_01064_gb300", "weights")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nmg.Context(0)


def items_spec():
    W = nmg.load_weights(os.path.join(WDIR, "c2_2d_n128_s2_a1e-2.npz"))
    # (n, levels, sigma, alpha, precision, batch); smoothers trained on the
    # sigma-2 operator serve every grid size (per-level operators coincide);
    # on the sigma-1 operator they diverge, which must also be reproduced
    # bit for bit
    return W, [(128, 5, 2.0, 1e-2, "bf16_refine", 6), (64, 4, 2.0, 1e-2, "bf16_refine", 9),
               (64, 4, 2.0, 1e-2, "fp32", 5), (32, 3, 1.0, 1e-2, "bf16fast_refine", 4)]


def build(ctx, W, spec, seed):
    out = []
    for k, (n, L, sg, al, prec, B) in enumerate(spec):
        taps = I.gaussian_taps(sg)
        G = nmg.Hierarchy(ctx, dim=2, n=n, levels=L, alpha=al, taps=taps, precision=prec,
                          weights=W)
        f, _ = I.rhs_2d_waves_rects(n, B, seed + k, sg)
        fd = torch.tensor(f, dtype=torch.float32, device="cuda")
        ud = torch.zeros(fd.shape, dtype=torch.float32 if prec == "fp32" else torch.float64,
                         device="cuda")
        out.append((G, fd, ud, taps))
    return out


@pytest.mark.parametrize("graphs", [True, False])
def test_multi_equals_alone(ctx, graphs):
    W, spec = items_spec()
    ctx.set_graphs(graphs)
    try:
        alone = build(ctx, W, spec, 500)
        res_alone = [G.solve(f, u, rtol=1e-6, max_cycles=80) for G, f, u, _ in alone]
        together = build(ctx, W, spec, 500)
        res_multi = nmg.solve_multi(ctx, [(G, f, u) for G, f, u, _ in together], rtol=1e-6,
                                    max_cycles=80)
    finally:
        ctx.set_graphs(True)
    for (Ga, fa, ua, _), (Gm, fm, um, _), ra, rm in zip(alone, together, res_alone, res_multi):
        assert np.array_equal(ra[0], rm[0])                       # cycles
        assert np.array_equal(ra[1], rm[1])                       # status
        iv = torch.int64 if ua.dtype == torch.float64 else torch.int32
        assert torch.equal(ua.view(iv), um.view(iv))              # iterates, bitwise (NaN-safe)
    # the sigma-2 items converge to 1e-6, checked with the oracle's own apply
    for (G, f, u, taps), (n, L, sg, al, prec, B), r in zip(together, spec, res_multi):
        if sg == 2.0:
            assert np.all(r[1] == 0)
            H = O.build_hierarchy_2d(taps, n, al, L)
            rr = O.relres(H, f.double().cpu().numpy(), u.double().cpu().numpy())
            assert np.all(rr <= (1.5e-6 if prec == "fp32" else 1.01e-6)), rr


def test_multi_rejects_duplicate_hierarchy(ctx):
    W, spec = items_spec()
    (G, f, u, _), = build(ctx, W, spec[:1], 1)
    with pytest.raises(nmg.NMGError):
        nmg.solve_multi(ctx, [(G, f, u), (G, f, u)])


MIX_SIZES, MIX_SIGMAS, MIX_ALPHAS = [64, 128, 256, 512], [1.0, 2.0, 4.0], [1e-3, 1e-2]


@pytest.fixture(scope="module")
def mixed_classes(ctx):
    """One right-hand side of each of the 24 operator classes of the mixed
    batch (sides 64..512, PSF sigma 1, 2, 4 px, alpha 1e-3 and 1e-2, levels
    log2(n) - 2), each with its class's trained smoothers."""
    from paper_2603_01064_gb300.weights import operator_weights
    out = []
    k = 0
    for n in MIX_SIZES:
        for sg in MIX_SIGMAS:
            for al in MIX_ALPHAS:
                L = int(np.log2(n)) - 2
                W = operator_weights(sg, al, L)
                taps = I.gaussian_taps(sg)
                G = nmg.Hierarchy(ctx, dim=2, n=n, levels=L, alpha=al, taps=taps,
                                  precision="bf16_refine", weights=W)
                f, _ = I.rhs_2d_waves_rects(n, 1, 900 + k, sg)
                out.append(dict(n=n, sigma=sg, alpha=al, L=L, W=W, taps=taps, G=G, f=f))
                k += 1
    return out


def _multi(ctx, classes, max_cycles):
    items = []
    for c in classes:
        fd = torch.tensor(c["f"], dtype=torch.float32, device="cuda")
        items.append((c["G"], fd, torch.zeros(fd.shape, dtype=torch.float64, device="cuda")))
    res = nmg.solve_multi(ctx, items, rtol=1e-6, max_cycles=max_cycles)
    torch.cuda.synchronize()
    return items, res


def test_mixed_classes_one_cycle_vs_oracle(ctx, mixed_classes):
    """All 24 classes in one multi-solve limited to one cycle: each item's
    iterate against the oracle's cycle from zero on its own hierarchy, at the
    bf16 form's per-cycle bar 1e-3 (max of norm-wise and element-wise)."""
    items, res = _multi(ctx, mixed_classes, 1)
    for c, (G, fd, ud), (cyc, st, rr) in zip(mixed_classes, items, res):
        assert cyc[0] == 1
        H = O.build_hierarchy_2d(c["taps"], c["n"], c["alpha"], c["L"])
        ref = O.nmgf(H, c["W"], 0, None, fd.double().cpu().numpy())
        err = float(np.max(rel_both(ud.cpu().numpy(), ref)))
        assert err < 1e-3, (c["n"], c["sigma"], c["alpha"], err)


def test_mixed_classes_solve_to_tolerance(ctx, mixed_classes):
    """All 24 classes solved together to 1e-6: every item converges and its
    iterate meets 1e-6 under the oracle's own apply."""
    items, res = _multi(ctx, mixed_classes, 250)
    for c, (G, fd, ud), (cyc, st, rr) in zip(mixed_classes, items, res):
        tag = (c["n"], c["sigma"], c["alpha"], int(cyc[0]), float(rr[0]))
        assert st[0] == nmg.CONVERGED, tag
        H = O.build_hierarchy_2d(c["taps"], c["n"], c["alpha"], c["L"])
        rr_o = O.relres(H, fd.double().cpu().numpy(), ud.cpu().numpy())
        assert rr_o[0] <= 1.01e-6, tag + (float(rr_o[0]),)
