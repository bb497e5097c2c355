"""Error measures of the GPU parity tests.

Per right-hand side, the norm-wise relative error ||a - b|| / ||b|| and the
element-wise relative error max |a - b| / max |b| (b the oracle's result).
Every bar is applied to the larger of the two, so one wrong grid point (a
halo pixel, a tile corner) that a norm would average away still fails.
"""
import numpy as np


def rel_both(a, b):
    """Per right-hand side max(norm-wise, element-wise) relative error."""
    a = np.asarray(a, np.float64).reshape(np.shape(a)[0], -1)
    b = np.asarray(b, np.float64).reshape(np.shape(b)[0], -1)
    d = a - b
    nw = np.linalg.norm(d, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)
    ew = np.abs(d).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)
    return np.maximum(nw, ew)
