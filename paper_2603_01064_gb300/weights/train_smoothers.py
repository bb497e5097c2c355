"""Offline level-wise training of the CNN smoothers (Algorithm 5).

This is the prerequisite that produces the frozen smoother weights the CUDA
solve path loads; it is not part of the solve path.  It is a self-contained
PyTorch program (CPU or GPU) with its own dense hierarchy:

* the cycle is NMGF1d / NMGF2d (Algorithms 3, 4) started from zero;
* level l is trained with the level-wise filtered loss of Eq. (6) (1D) /
  Eq. (9) (2D): the fine-grid error left after the filtered corrections of
  levels 1..l-1 and the *unfiltered* prolonged output of level l, weighted by
  the fine-grid mask m_l (Section 3.2);
* only theta_l receives the gradient of L_l (Algorithm 5's update line);
  outputs of earlier levels enter L_l as constants;
* training pairs come from DataGeneration (Algorithm 5): a random error x,
  y = A x, then k ~ U{1..K} no-grad cycles replacing (x, y) by
  (x - c, A (x - c)) with c = NMGF(0, y);
* Adam (Section 3.4), optional curriculum over alpha (Section 4.1.1): the
  nets trained for a larger alpha initialise the next smaller one.

Training choices the paper leaves open (documented with the weights):
random errors are a mix of white noise and Gaussian-correlated noise with a
random correlation length; each sample is scaled to unit error norm after
the rollouts so that all rollout depths weigh equally (the smoother is
positively homogeneous, so this does not change what it has to learn).

Usage:
  python -m paper_2603_01064_gb300.weights.train_smoothers --config c2 --out c2_2d_sigma2_a1e-2.npz
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np
import torch
import torch.nn as nn
import torch.nn.functional as F

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(os.path.dirname(_HERE))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)
import nmg_inputs  # noqa: E402  (seeded problem data only)


# ---------------------------------------------------------------------------
# networks
# ---------------------------------------------------------------------------

class CNN(nn.Module):
    """conv -> ReLU -> ... -> conv, zero 'same' padding, bias on every layer.

    `gain` is a fixed output scale used only during training (the smoother has
    to amplify high frequencies by about 1/alpha); it is folded into the last
    layer's weight and bias on export, so the exported net is the plain CNN.
    """

    def __init__(self, dim, layers, width, ksize, gain=1.0):
        super().__init__()
        Conv = nn.Conv1d if dim == 1 else nn.Conv2d
        chans = [1] + [width] * (layers - 1) + [1]
        self.convs = nn.ModuleList(
            Conv(chans[i], chans[i + 1], ksize, padding=ksize // 2) for i in range(layers))
        self.gain = gain
        # zero last layer: the untrained cycle is the pure coarse correction
        nn.init.zeros_(self.convs[-1].weight)
        nn.init.zeros_(self.convs[-1].bias)

    def forward(self, x):
        z = x.unsqueeze(1)
        for i, c in enumerate(self.convs):
            z = c(z)
            if i < len(self.convs) - 1:
                z = F.relu(z)
        return self.gain * z.squeeze(1)


class FNO(nn.Module):
    """2D FNO smoother of Appendix A: pointwise lift 1 -> width, `layers`
    Fourier layers z <- ReLU(W * z + B + DFT^-1(R . DFT(z))) with R on the
    modes k1 in [0, m) and [n - m, n), k2 in [0, m) of the real 2D DFT, and a
    pointwise projection width -> 1 (times the training gain, folded into the
    projection on export)."""

    def __init__(self, layers, width, ksize, modes, gain=1.0):
        super().__init__()
        self.m = modes
        self.lift = nn.Conv2d(1, width, 1)
        self.w = nn.ModuleList(nn.Conv2d(width, width, ksize, padding=ksize // 2)
                               for _ in range(layers))
        # R starts near zero: the untrained layer is its local W term, and
        # the spectral part grows from there
        scale = 0.01 / width
        self.r = nn.ParameterList(
            nn.Parameter(scale * torch.randn(2, width, width, modes, modes, dtype=torch.cfloat))
            for _ in range(layers))
        self.proj = nn.Conv2d(width, 1, 1)
        self.gain = gain
        nn.init.zeros_(self.proj.weight)
        nn.init.zeros_(self.proj.bias)

    def spectral(self, z, R):
        n, m = z.shape[-1], self.m
        Z = torch.fft.rfft2(z)
        Y = torch.zeros(z.shape[0], R.shape[2], n, n // 2 + 1, dtype=Z.dtype, device=z.device)
        Y[:, :, :m, :m] = torch.einsum("bixy,ioxy->boxy", Z[:, :, :m, :m], R[0])
        Y[:, :, n - m:, :m] = torch.einsum("bixy,ioxy->boxy", Z[:, :, n - m:, :m], R[1])
        return torch.fft.irfft2(Y, s=(n, n))

    def forward(self, x):
        z = self.lift(x.unsqueeze(1))
        for W, R in zip(self.w, self.r):
            z = F.relu(W(z) + self.spectral(z, R))
        return self.gain * self.proj(z).squeeze(1)


# ---------------------------------------------------------------------------
# dense hierarchy (same definitions as the solve path; written independently)
# ---------------------------------------------------------------------------

def _prolong_np(nc):
    P = np.zeros((2 * nc, nc))
    for J in range(nc):
        P[2 * J, J] = 1.0
        P[2 * J + 1, J] = 0.5
        if J > 0:
            P[2 * J - 1, J] = 0.5
    return P


class Problem:
    def __init__(self, dim, n, levels, alpha, taps=None, col=None, device="cpu",
                 dtype=torch.float32, reg=None):
        self.dim, self.n, self.L, self.alpha = dim, n, levels, alpha
        self.device, self.dtype = device, dtype
        T = lambda a: torch.tensor(a, dtype=dtype, device=device)  # noqa: E731
        self.P, self.R = [], []
        for l in range(levels - 1):
            P = _prolong_np((n >> l) // 2)
            self.P.append(T(P))
            self.R.append(T(P.T / 2.0))
        if dim == 1:
            i = np.arange(n)
            # A = hK + alpha D: D = I (Tikhonov) or the anisotropic
            # tridiagonal of Section 4.1, given as (diag, off)
            D = np.eye(n) if reg is None else (np.diag(reg[0]) + np.diag(reg[1], 1) +
                                               np.diag(reg[1], -1))
            A = col[np.abs(i[:, None] - i[None, :])] + alpha * D
            ops = [A]
            for l in range(levels - 1):
                P = _prolong_np((n >> l) // 2)
                A = (P.T / 2.0) @ A @ P
                ops.append(A)
            self.A = [T(a) for a in ops]
            self.A64 = torch.tensor(ops[0], dtype=torch.float64, device=device)
            coarse = ops[-1]
        else:
            w = len(taps) - 1
            i = np.arange(n)
            d = np.abs(i[:, None] - i[None, :])
            K = np.where(d <= w, taps[np.minimum(d, w)], 0.0)
            M = np.eye(n)
            Ms, Ks = [M], [K]
            for l in range(levels - 1):
                P = _prolong_np((n >> l) // 2)
                M = (P.T / 2.0) @ M @ P
                K = (P.T / 2.0) @ K @ P
                Ms.append(M)
                Ks.append(K)
            self.M = [T(a) for a in Ms]
            self.K = [T(a) for a in Ks]
            self.M64 = torch.tensor(Ms[0], dtype=torch.float64, device=device)
            self.K64 = torch.tensor(Ks[0], dtype=torch.float64, device=device)
            coarse = alpha * np.kron(Ms[-1], Ms[-1]) + np.kron(Ks[-1], Ks[-1])
        self.coarse_inv = T(np.linalg.inv(coarse))
        # output filter masks m'_l (local symbol, the same on every level)
        self.fmask = []
        for l in range(levels - 1):
            m = n >> l
            j = np.arange(m)
            w_ = 2 * np.pi * np.minimum(j, m - j) / m
            mk = np.sqrt(w_ / np.pi) if dim == 1 else np.sqrt(np.maximum(w_[:, None], w_[None, :]) / np.pi)
            self.fmask.append(T(mk))
        # loss masks m_l on the finest grid
        j = np.arange(n)
        wf = 2 * np.pi * np.minimum(j, n - j) / n
        wmax = wf if dim == 1 else np.maximum(wf[:, None], wf[None, :])
        self.lmask = []
        for l in range(levels - 1):
            band = np.pi / (1 << l)
            self.lmask.append(T(np.where(wmax <= band, np.sqrt(wmax / band), 0.0)))

    def top_gain(self, l):
        """1 / Rayleigh quotient of A_l at the highest-frequency mode."""
        m = self.n >> l
        sgn = torch.tensor([(-1.0) ** i for i in range(m)], dtype=self.dtype, device=self.device)
        v = sgn if self.dim == 1 else sgn[:, None] * sgn[None, :]
        v = v.unsqueeze(0)
        return float((v * v).sum() / (v * self.apply(l, v)).sum())

    def apply(self, l, x):
        if self.dim == 1:
            return x @ self.A[l].T
        return self.alpha * (self.M[l] @ x @ self.M[l].T) + self.K[l] @ x @ self.K[l].T

    def apply64(self, x):
        """The fine-level operator in fp64 (the outer residual of evaluate)."""
        if self.dim == 1:
            return x @ self.A64.T
        return self.alpha * (self.M64 @ x @ self.M64.T) + self.K64 @ x @ self.K64.T

    def restrict(self, l, r):
        R = self.R[l]
        return r @ R.T if self.dim == 1 else R @ r @ R.T

    def prolong(self, l, e):
        P = self.P[l]
        return e @ P.T if self.dim == 1 else P @ e @ P.T

    def to_fine(self, l, v):
        for k in range(l - 1, -1, -1):
            v = self.prolong(k, v)
        return v

    def filt(self, l, h):
        if self.dim == 1:
            return torch.fft.ifft(self.fmask[l] * torch.fft.fft(h)).real
        return torch.fft.ifft2(self.fmask[l] * torch.fft.fft2(h)).real

    def coarse_solve(self, y):
        B = y.shape[0]
        return (y.reshape(B, -1) @ self.coarse_inv.T).reshape(y.shape)


def _norm(v):
    return v.reshape(v.shape[0], -1).norm(dim=1).reshape((-1,) + (1,) * (v.dim() - 1))


def smooth(net, b):
    s = _norm(b)
    safe = torch.where(s > 0, s, torch.ones_like(s))
    return net(b / safe) * safe


def cycle(prob, nets, l, y, xstar=None):
    """NMGF(x*, y) at level l (Algorithms 3/4)."""
    if l == prob.L - 1:
        return prob.coarse_solve(y)
    b = y if xstar is None else y - prob.apply(l, xstar)
    h = smooth(nets[l], b)
    x = prob.filt(l, h) if xstar is None else xstar + prob.filt(l, h)
    yc = prob.restrict(l, y - prob.apply(l, x))
    return x + prob.prolong(l, cycle(prob, nets, l + 1, yc))


# ---------------------------------------------------------------------------
# data generation (Algorithm 5) and the level-wise loss (Eqs. (6), (9))
# ---------------------------------------------------------------------------

def random_errors(prob, bs, gen):
    shape = (bs, prob.n) if prob.dim == 1 else (bs, prob.n, prob.n)
    x = torch.randn(shape, generator=gen, dtype=prob.dtype)
    # half of the samples: correlated noise with a random correlation length
    for i in range(bs // 2):
        ell = float(torch.exp(torch.rand(1, generator=gen, dtype=torch.float64) * math.log(16.0)))
        w = int(math.ceil(3 * ell))
        t = torch.arange(-w, w + 1, dtype=prob.dtype)
        g = torch.exp(-t * t / (2 * ell * ell))
        g = g / g.norm()
        v = x[i:i + 1].unsqueeze(1)
        if prob.dim == 1:
            v = F.conv1d(v, g.view(1, 1, -1), padding=w)
        else:
            v = F.conv2d(v, g.view(1, 1, 1, -1), padding=(0, w))
            v = F.conv2d(v, g.view(1, 1, -1, 1), padding=(w, 0))
        x[i] = v[0, 0]
    return x.to(prob.device)


@torch.no_grad()
def data_generation(prob, nets, bs, K, gen):
    x = random_errors(prob, bs, gen)
    y = prob.apply(0, x)
    ks = torch.randint(1, K + 1, (bs,), generator=gen)
    for j in range(1, K + 1):
        idx = torch.nonzero(ks >= j).flatten().to(prob.device)
        if idx.numel() == 0:
            break
        c = cycle(prob, nets, 0, y[idx])
        xn = x[idx] - c
        sn = _norm(xn)
        sn = torch.where(sn > 0, sn, torch.ones_like(sn))
        xn = xn / sn
        x[idx] = xn
        y[idx] = prob.apply(0, xn)
    s = _norm(x)
    s = torch.where(s > 0, s, torch.ones_like(s))
    return x / s, y / s


def levelwise_losses(prob, nets, x, y):
    """One cycle from zero; L_l for each smoother level l."""
    losses = []
    corr = torch.zeros_like(x)
    yl = y
    dims = (-1,) if prob.dim == 1 else (-2, -1)
    for l in range(prob.L - 1):
        b = yl.detach()
        h = smooth(nets[l], b)
        e = x - corr - prob.to_fine(l, h)
        E = torch.fft.fftn(e, dim=dims, norm="ortho")
        losses.append((prob.lmask[l] * E).abs().pow(2).reshape(x.shape[0], -1).sum(1).mean())
        hf = prob.filt(l, h.detach())
        corr = corr + prob.to_fine(l, hf)
        yl = prob.restrict(l, yl - prob.apply(l, hf))
    return losses


@torch.no_grad()
def evaluate(prob, nets, f, rtol=1e-6, max_cycles=60):
    """The outer iteration x^t = NMGF(x^{t-1}, f) from zero (Section 3.2) as
    the library's refinement forms run it: u and the residual r = f - A u in
    fp64, the cycle (in the problem's precision) on r from zero, its result
    added to u in fp64.  (A cycle run wholly in fp32 stalls at a few 1e-6 on
    the small-alpha operators, so it would hide whether a set converges.)
    Returns per-RHS cycles to rtol (max_cycles + 1 if not) and the largest
    relative residual after each cycle."""
    f64 = f.double()
    u = torch.zeros_like(f64)
    fn = _norm(f64).flatten()
    cyc = torch.full((f.shape[0],), max_cycles + 1, device=f.device)
    hist = []
    for t in range(1, max_cycles + 1):
        r = f64 - prob.apply64(u)
        u = u + cycle(prob, nets, 0, r.to(prob.dtype)).double()
        rr = (_norm(f64 - prob.apply64(u)).flatten() / fn)
        hist.append(rr.max().item())
        newly = (rr <= rtol) & (cyc > max_cycles)
        cyc[newly] = t
        if (cyc <= max_cycles).all():
            break
    return cyc, hist


def nets_to_npz(nets, path, meta):
    arrs = {}
    for l, net in enumerate(nets):
        last = len(net.convs) - 1
        for i, c in enumerate(net.convs):
            g = net.gain if i == last else 1.0
            arrs[f"l{l}_w{i}"] = g * c.weight.detach().cpu().double().numpy()
            arrs[f"l{l}_b{i}"] = g * c.bias.detach().cpu().double().numpy()
        # The output layer's bias adds a constant to h, and the cycle only
        # uses F'(h): the mask is zero at zero frequency, so the constant
        # never reaches the iterate.  Left in, it can grow far larger than
        # the filtered part (it sets ||h|| / ||F'h||, the factor by which
        # rounding in the smoother is amplified in the cycle's result), so
        # it is dropped on export; the filtered cycle is unchanged.
        arrs[f"l{l}_b{last}"] = np.zeros_like(arrs[f"l{l}_b{last}"])
    for k, v in meta.items():
        arrs["meta_" + k] = np.array(v)
    np.savez(path, **arrs)


def fno_to_npz(nets, path, meta):
    """Export FNO smoothers: l{l}_lift_w [c], l{l}_lift_b [c], l{l}_k{i}_w
    [c, c, k, k], l{l}_k{i}_b [c], l{l}_k{i}_rre / _rim [2, c, c, m, m],
    l{l}_proj_w [c], l{l}_proj_b [1] (gain folded in; the projection's bias
    exported as zero for the reason given in nets_to_npz).  Stored as fp32,
    the precision the net was trained in."""
    arrs = {}
    np_ = lambda t: t.detach().cpu().numpy().astype(np.float32)  # noqa: E731
    for l, net in enumerate(nets):
        arrs[f"l{l}_lift_w"] = np_(net.lift.weight).reshape(-1)
        arrs[f"l{l}_lift_b"] = np_(net.lift.bias)
        for i, (W, R) in enumerate(zip(net.w, net.r)):
            arrs[f"l{l}_k{i}_w"] = np_(W.weight)
            arrs[f"l{l}_k{i}_b"] = np_(W.bias)
            arrs[f"l{l}_k{i}_rre"] = np_(R.real)
            arrs[f"l{l}_k{i}_rim"] = np_(R.imag)
        arrs[f"l{l}_proj_w"] = (net.gain * np_(net.proj.weight)).reshape(-1)
        arrs[f"l{l}_proj_b"] = np.zeros(1, np.float32)
    for k, v in meta.items():
        arrs["meta_" + k] = np.array(v)
    arrs["meta_arch"] = np.array("fno")
    np.savez(path, **arrs)


def nets_from_npz(path, dim, layers, width, ksize, device="cpu", gains=None, depths=None):
    """CNN smoothers from a stored file (gains as used in training).  A level
    whose stored depth differs from depths[l] (when given) starts from a fresh
    net of that depth instead."""
    z = np.load(path)
    nl = int(z["meta_smoother_levels"])
    nets = []
    for l in range(nl):
        g = 1.0 if gains is None else gains[l]
        stored = len([k for k in z.files if k.startswith(f"l{l}_w")])
        want = stored if depths is None else depths[l]
        net = CNN(dim, want, width, ksize, gain=g)
        if want != stored:
            print(f"level {l}: stored depth {stored}, fresh net of depth {want}")
            nets.append(net.to(device))
            continue
        last = len(net.convs) - 1
        for i, c in enumerate(net.convs):
            s = 1.0 / g if i == last else 1.0
            c.weight.data = torch.tensor(s * z[f"l{l}_w{i}"], dtype=torch.float32)
            c.bias.data = torch.tensor(s * z[f"l{l}_b{i}"], dtype=torch.float32)
        nets.append(net.to(device))
    return nets


PRESETS = {
    # dim, n, levels, alpha, kernel, batch, epochs
    "c1": dict(dim=1, n=256, levels=3, alpha=1e-3, width_t=0.05, layers=3, width=16, ksize=5),
    # the anisotropic regularisation of Section 4.1 (A = alpha D + hK)
    "c1a": dict(dim=1, n=256, levels=3, alpha=1e-5, width_t=0.05, layers=3, width=16, ksize=5,
                reg="aniso"),
    "c2": dict(dim=2, n=128, levels=5, alpha=1e-2, sigma=2.0, layers=4, width=32, ksize=3),
    "c3": dict(dim=2, n=512, levels=7, alpha=1e-3, sigma=4.0, layers=4, width=32, ksize=3,
               rhs="waves"),
    # the FNO smoother of Appendix A on the 128x128 operator (8 modes: the
    # most the 16x16 coarsest smoother level holds)
    "c2f": dict(dim=2, n=128, levels=5, alpha=1e-2, sigma=2.0, layers=4, width=32, ksize=3,
                arch="fno", modes=8),
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--sigma", type=float, default=None)
    ap.add_argument("--epochs", type=int, default=1500)
    ap.add_argument("--bs", type=int, default=20)
    ap.add_argument("--K", type=int, default=10)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--init", default=None, help="npz to initialise from (curriculum)")
    ap.add_argument("--device", default="cpu")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--eval-batch", type=int, default=8)
    ap.add_argument("--eval-every", type=int, default=100)
    ap.add_argument("--eval-cycles", type=int, default=60,
                    help="cycle limit of the evaluation solves")
    ap.add_argument("--depths", default=None,
                    help="comma list of CNN layers per smoother level (default: the preset's "
                         "layers on every level)")
    ap.add_argument("--train-levels", default=None,
                    help="comma list of smoother levels to train (default: all); the others "
                         "stay as initialised")
    ap.add_argument("--clip", type=float, default=0.0,
                    help="clip each trained level's gradient norm to this (0: off)")
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    if a.threads:
        torch.set_num_threads(a.threads)
    cfg = dict(PRESETS[a.config])
    for k in ("n", "levels", "alpha", "sigma"):
        if getattr(a, k) is not None:
            cfg[k] = getattr(a, k)
    torch.manual_seed(a.seed)
    gen = torch.Generator().manual_seed(a.seed)
    dim = cfg["dim"]
    if dim == 1:
        col = nmg_inputs.kernel_column_1d(cfg["n"], cfg["width_t"])
        reg = nmg_inputs.aniso_regularisation_1d(cfg["n"]) if cfg.get("reg") == "aniso" else None
        prob = Problem(1, cfg["n"], cfg["levels"], cfg["alpha"], col=col, device=a.device,
                       reg=reg)
    else:
        taps = nmg_inputs.gaussian_taps(cfg["sigma"])
        prob = Problem(2, cfg["n"], cfg["levels"], cfg["alpha"], taps=taps, device=a.device)
    gains = [prob.top_gain(l) for l in range(cfg["levels"] - 1)]
    print("output gains", ["%.3g" % g for g in gains])
    nsm = cfg["levels"] - 1
    depths = [cfg["layers"]] * nsm if a.depths is None else [int(v) for v in a.depths.split(",")]
    if len(depths) != nsm or min(depths) < 2:
        raise SystemExit(f"--depths needs {nsm} entries >= 2")
    if cfg.get("arch") == "fno":
        nets = [FNO(cfg["layers"], cfg["width"], cfg["ksize"], cfg["modes"], gain=g).to(a.device)
                for g in gains]
    elif a.init:
        nets = nets_from_npz(a.init, dim, cfg["layers"], cfg["width"], cfg["ksize"], a.device, gains,
                             depths if a.depths is not None else None)
    else:
        nets = [CNN(dim, d, cfg["width"], cfg["ksize"], gain=g).to(a.device)
                for d, g in zip(depths, gains)]
    if cfg.get("arch") != "fno":
        cfg["depths"] = [len(n_.convs) for n_ in nets]
    train = list(range(nsm)) if a.train_levels is None else [int(v) for v in a.train_levels.split(",")]
    for l, n_ in enumerate(nets):
        n_.requires_grad_(l in train)
    opts = [torch.optim.Adam(nets[l].parameters(), lr=a.lr) for l in train]
    scheds = [torch.optim.lr_scheduler.CosineAnnealingLR(o, a.epochs, eta_min=a.lr * 0.02) for o in opts]
    if dim == 1:
        f_eval, _ = nmg_inputs.rhs_1d_sines_steps(cfg["n"], a.eval_batch, 4242)
    elif cfg.get("rhs") == "waves":
        f_eval, _ = nmg_inputs.rhs_2d_waves_rects(cfg["n"], a.eval_batch, 4242, cfg["sigma"])
    else:
        f_eval, _ = nmg_inputs.rhs_2d_ellipses_grf(cfg["n"], a.eval_batch, 4242, cfg["sigma"])
    f_eval = torch.tensor(f_eval, dtype=torch.float32, device=a.device)
    t0 = time.time()
    best = float("inf")
    if a.epochs == 0:
        # evaluation only (the initial nets, e.g. a stored file given by --init)
        cyc, hist = evaluate(prob, nets, f_eval, rtol=1e-6, max_cycles=a.eval_cycles)
        print(f"   eval cycles to 1e-6: {cyc.tolist()} relres every 10 cycles " +
              " ".join(f"{v:.1e}" for v in hist[9::10]), flush=True)
        return
    for ep in range(1, a.epochs + 1):
        x, y = data_generation(prob, nets, a.bs, a.K, gen)
        losses = levelwise_losses(prob, nets, x, y)
        for o in opts:
            o.zero_grad(set_to_none=True)
        sum(losses[l] for l in train).backward()
        if a.clip > 0:
            for l in train:
                torch.nn.utils.clip_grad_norm_(nets[l].parameters(), a.clip)
        for o, s in zip(opts, scheds):
            o.step()
            s.step()
        if ep % 50 == 0 or ep == 1:
            print(f"ep {ep} t={time.time() - t0:.0f}s losses " +
                  " ".join(f"{v.item():.3e}" for v in losses), flush=True)
        if ep % a.eval_every == 0 or ep == a.epochs:
            cyc, hist = evaluate(prob, nets, f_eval, rtol=1e-6, max_cycles=a.eval_cycles)
            # mean cycles to 1e-6; if some right-hand side did not get there,
            # also the orders of magnitude left (so checkpoints that do not
            # converge within the limit are still ranked by how far they got)
            score = float(cyc.double().mean())
            if hist and hist[-1] > 1e-6:
                score += 100.0 * math.log10(hist[-1] / 1e-6)
            print(f"   eval cycles to 1e-6: {cyc.tolist()} last relres {hist[-1]:.2e}", flush=True)
            if score <= best:
                # keep the checkpoint that solves the evaluation set in the fewest cycles
                best = score
                meta = dict(cfg, epochs=ep, bs=a.bs, K=a.K, lr=a.lr, seed=a.seed,
                            smoother_levels=cfg["levels"] - 1, eval_cycles=score)
                (fno_to_npz if cfg.get("arch") == "fno" else nets_to_npz)(nets, a.out, meta)
                print(f"   saved (mean cycles {score:.2f})", flush=True)
    print("done", a.out, f"{time.time() - t0:.0f}s")


if __name__ == "__main__":
    main()
