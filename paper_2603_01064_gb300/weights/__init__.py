"""Trained smoother sets shipped with the package, and the table of which
set serves which operator class."""
import os

WEIGHTS_DIR = os.path.dirname(os.path.abspath(__file__))

# CNN smoother sets per operator class (PSF sigma in px, alpha), each trained
# level-wise (Algorithm 5) on one grid.  The Galerkin level operators of a
# class depend on the level index, not on the grid side, so a set serves
# every side of its class; a hierarchy with more smoother levels than the
# set repeats the set's last (coarsest) net.
OPERATOR_WEIGHTS = {
    (1.0, 1e-2): "mix_2d_n256_s1_a1e-2.npz", (1.0, 1e-3): "mix_2d_n256_s1_a1e-3.npz",
    (2.0, 1e-2): "mix_2d_n512_s2_a1e-2.npz", (2.0, 1e-3): "mix_2d_n512_s2_a1e-3.npz",
    (4.0, 1e-2): "c3_2d_n512_s4_a1e-2.npz", (4.0, 1e-3): "c3_2d_n512_s4_a1e-3.npz",
    (8.0, 1e-2): "mix_2d_n512_s8_a1e-2.npz", (8.0, 1e-3): "mix_2d_n512_s8_a1e-3.npz",
}


def operator_weights(sigma, alpha, levels):
    """The smoother set of an operator class, cut or extended to levels - 1
    smoother levels."""
    from .. import load_weights
    W = load_weights(os.path.join(WEIGHTS_DIR, OPERATOR_WEIGHTS[(float(sigma), float(alpha))]))
    return [W[min(l, len(W) - 1)] for l in range(levels - 1)]
