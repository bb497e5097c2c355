"""The offline level-wise trainer (Algorithm 5) on the CPU, at toy sizes.

* Its own cycle (a separate PyTorch implementation of Algorithms 3/4 with a
  dense hierarchy) equals the FP64 oracle's cycle for the same weights, with
  and without the exported zero output bias (F' removes constants, so the
  filtered cycle does not depend on it).
* DataGeneration returns pairs with y = A x and unit error norms.
* A few Adam steps on the level-wise loss of level 0 lower it.
* Export to npz and the library's loader round-trip the weights.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import nmg_inputs as I  # noqa: E402
import oracle as O  # noqa: E402
import paper_2603_01064_gb300 as nmg  # noqa: E402
from paper_2603_01064_gb300.weights import train_smoothers as T  # noqa: E402

N, L, ALPHA, SIGMA = 16, 3, 1e-2, 1.0


def _nets(seed, dim=2, layers=4, width=8, ksize=3):
    torch.manual_seed(seed)
    nets = []
    for _ in range(L - 1):
        net = T.CNN(dim, layers, width, ksize).double()
        with torch.no_grad():  # the trainer zero-initialises the output layer
            net.convs[-1].weight.normal_(0.0, 0.3)
            net.convs[-1].bias.normal_(0.0, 0.3)
        nets.append(net)
    return nets


def _weights(nets, zero_out_bias):
    W = []
    for net in nets:
        lv = [(c.weight.detach().numpy().copy(), c.bias.detach().numpy().copy()) for c in net.convs]
        if zero_out_bias:
            lv[-1] = (lv[-1][0], np.zeros_like(lv[-1][1]))
        W.append(lv)
    return W


def _problem():
    return T.Problem(2, N, L, ALPHA, taps=I.gaussian_taps(SIGMA), dtype=torch.float64)


@pytest.mark.parametrize("zero_out_bias", [False, True])
def test_trainer_cycle_equals_oracle_cycle(zero_out_bias):
    nets = _nets(0)
    prob = _problem()
    y = np.random.default_rng(1).standard_normal((3, N, N))
    with torch.no_grad():
        xt = T.cycle(prob, nets, 0, torch.tensor(y)).numpy()
    H = O.build_hierarchy_2d(I.gaussian_taps(SIGMA), N, ALPHA, L)
    xo = O.nmgf(H, _weights(nets, zero_out_bias), 0, None, y)
    assert np.max(np.abs(xt - xo)) <= 1e-11 * np.max(np.abs(xo))


def test_evaluation_is_the_refined_outer_iteration():
    """The trainer's evaluation runs x^t = NMGF(x^{t-1}, f) with the residual
    and update in fp64 around its fp32 cycle: its residual history over
    three cycles equals the FP64 oracle's iteration to fp32 rounding."""
    nets = _nets(0)
    W = _weights(nets, False)
    nets32 = [n.float() for n in nets]
    prob = T.Problem(2, N, L, ALPHA, taps=I.gaussian_taps(SIGMA), dtype=torch.float32)
    f = np.random.default_rng(5).standard_normal((2, N, N)).astype(np.float32)
    cyc, hist = T.evaluate(prob, nets32, torch.tensor(f), rtol=0.0, max_cycles=3)
    H = O.build_hierarchy_2d(I.gaussian_taps(SIGMA), N, ALPHA, L)
    f64 = f.astype(np.float64)
    u = np.zeros_like(f64)
    for t in range(3):
        u = O.nmgf(H, W, 0, u, f64)
        rr = np.max(O.relres(H, f64, u))
        assert abs(hist[t] - rr) <= 1e-4 * rr, (t, hist[t], rr)


def test_data_generation_pairs():
    nets = _nets(1)
    prob = _problem()
    gen = torch.Generator().manual_seed(2)
    x, y = T.data_generation(prob, nets, 6, 3, gen)
    assert torch.allclose(y, prob.apply(0, x), atol=1e-12)
    assert torch.allclose(x.reshape(6, -1).norm(dim=1), torch.ones(6, dtype=torch.float64))


def test_levelwise_loss_decreases_with_adam():
    torch.manual_seed(3)
    prob = T.Problem(2, N, L, ALPHA, taps=I.gaussian_taps(SIGMA))
    nets = [T.CNN(2, 4, 8, 3, gain=prob.top_gain(l)) for l in range(L - 1)]
    gen = torch.Generator().manual_seed(4)
    x, y = T.data_generation(prob, nets, 16, 2, gen)
    opt = torch.optim.Adam(nets[0].parameters(), lr=1e-3)  # the trainer's default rate
    first = None
    for _ in range(40):
        loss = T.levelwise_losses(prob, nets, x, y)[0]
        if first is None:
            first = loss.item()
        opt.zero_grad()
        loss.backward()
        opt.step()
    assert T.levelwise_losses(prob, nets, x, y)[0].item() < 0.85 * first


def test_export_round_trip(tmp_path):
    nets = [n.float() for n in _nets(5)]
    for n_, g in zip(nets, (2.0, 3.0)):
        n_.gain = g
    path = os.path.join(tmp_path, "w.npz")
    T.nets_to_npz(nets, path, {"smoother_levels": L - 1})
    W = nmg.load_weights(path)
    assert len(W) == L - 1 and all(len(lv) == 4 for lv in W)
    for lv, net in zip(W, nets):
        for i, (w, b) in enumerate(lv):
            g = net.gain if i == 3 else 1.0
            assert np.array_equal(w, g * net.convs[i].weight.detach().double().numpy())
            if i < 3:
                assert np.array_equal(b, net.convs[i].bias.detach().double().numpy())
            else:
                assert not np.any(b)  # output bias exported as zero


def test_trainer_command_line_writes_loadable_weights(tmp_path, capsys):
    """The trainer's entry point at a toy size: two epochs, an evaluation,
    and a weight file the library's loader reads (CNN, 2D and 1D)."""
    for cfg, extra in (("c2", ["--n", "16", "--levels", "3"]),
                       ("c1", ["--n", "32", "--levels", "2"])):
        out = os.path.join(tmp_path, cfg + ".npz")
        T.main(["--config", cfg, *extra, "--epochs", "2", "--bs", "2", "--K", "1",
                "--eval-batch", "1", "--eval-every", "1", "--out", out])
        W = nmg.load_weights(out)
        levels = int(extra[-1])
        assert len(W) == levels - 1
        dim = 2 if cfg == "c2" else 1
        assert all(np.asarray(w).ndim == 2 + dim for lv in W for (w, _) in lv)
    assert "saved" in capsys.readouterr().out
