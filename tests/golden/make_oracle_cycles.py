"""Write oracle_cycles.json: the number of cycles the FP64 oracle takes to
reach relative residual 1e-6 on the first right-hand side of each benchmark
workload (the outer iteration x^tau = NMGF(x^{tau-1}, f) from x^0 = 0 of
Section 3.2, the cycle of Algorithm 4).

The bench's CPU baseline and its reference arm time a bounded number of
oracle cycles and scale by this count, because a whole 512 x 512 solve on
the host takes minutes.  This script runs only the oracle (and reads the
stored smoother weights and the seeded input generators):

  python tests/golden/make_oracle_cycles.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import nmg_inputs as I  # noqa: E402
import oracle as O  # noqa: E402

WDIR = os.path.join(ROOT, "paper_2603_01064_gb300", "weights")

# (workload name, n, levels, alpha, sigma px, generator, seed, weight file)
WORKLOADS = [
    ("2d_bttb_512x512_sigma4_alpha1e-2_L7_batch64", 512, 7, 1e-2, 4.0, "waves_rects", 1003,
     "c3_2d_n512_s4_a1e-2.npz"),
    ("2d_bttb_128x128_sigma2_alpha1e-2_L5_batch256", 128, 5, 1e-2, 2.0, "ellipses_grf", 1002,
     "c2_2d_n128_s2_a1e-2.npz"),
]


def cnn_weights(path):
    """The stored CNN smoother file: arrays l{level}_w{layer}, l{level}_b{layer}."""
    z = np.load(path)
    nl = int(z["meta_smoother_levels"])
    nlayers = len([k for k in z.files if k.startswith("l0_w")])
    return [[(z[f"l{l}_w{i}"], z[f"l{l}_b{i}"]) for i in range(nlayers)] for l in range(nl)]


def main():
    out = {}
    for name, n, L, alpha, sigma, gen, seed, wfile in WORKLOADS:
        if gen == "waves_rects":
            f, _ = I.rhs_2d_waves_rects(n, 1, seed, sigma)
        else:
            f, _ = I.rhs_2d_ellipses_grf(n, 1, seed, sigma)
        H = O.build_hierarchy_2d(I.gaussian_taps(sigma), n, alpha, L)
        W = cnn_weights(os.path.join(WDIR, wfile))
        _, cyc, rr = O.solve(H, W, f, rtol=1e-6, max_cycles=100)
        out[name] = {"cycles": int(np.asarray(cyc).reshape(-1)[0]),
                     "relres": float(np.asarray(rr).reshape(-1)[0]),
                     "rhs": f"first right-hand side of the seeded generator {gen} (seed {seed}, "
                            "batch of 1)", "weights": wfile, "rtol": 1e-6}
        print(name, out[name], flush=True)
    with open(os.path.join(HERE, "oracle_cycles.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
