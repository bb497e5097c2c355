"""GB300 neural multigrid solver for convolution-type integral equations.

A thin ctypes binding over the C ABI in ``include/nmg.h`` (library
``_build/libnmg.so``, built by ``build.py``).  Every step of the solve runs in
the library's CUDA kernels; this module only marshals arguments (torch
tensors' device pointers, numpy host arrays) and raises on error codes.
There is no CPU fallback: importing works without the library, but creating
a ``Context`` fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

__all__ = [
    "FP64", "FP32", "BF16_REFINE", "BF16FAST_REFINE", "FP16_REFINE", "BF16X3_REFINE",
    "BF16TOP_REFINE", "PRECISIONS", "NMGError", "Context", "Hierarchy",
    "lib", "lib_path", "pack_weights", "load_weights", "SolveInfo", "solve_multi", "Server",
    "NOALLOC_SCRATCH_BYTES",
]

FP64, FP32, BF16_REFINE, BF16FAST_REFINE, FP16_REFINE, BF16X3_REFINE, BF16TOP_REFINE = \
    0, 1, 2, 3, 4, 5, 6
# kernel classes of Context.profile_read (NMG_K_* in nmg.h)
KERNEL_CLASSES = ["residual", "restrict", "cnn_first", "cnn_hidden", "cnn_last", "filter",
                  "coarse", "prolong", "refine_residual", "other", "cnn_fused"]
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16_refine": BF16_REFINE,
              "bf16fast_refine": BF16FAST_REFINE, "fp16_refine": FP16_REFINE,
              "bf16x3_refine": BF16X3_REFINE, "bf16top_refine": BF16TOP_REFINE}
CONVERGED, NOT_CONVERGED, DIVERGED = 0, 1, 2
NOALLOC_SCRATCH_BYTES = 1 << 20  # NMG_NOALLOC_SCRATCH_BYTES in nmg.h

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libnmg.so")
_lib = None


class NMGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nmg error {code}: {msg}")
        self.code = code


class _OpDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("levels", ctypes.c_int),
                ("alpha", ctypes.c_double), ("ntaps", ctypes.c_int),
                ("taps", ctypes.POINTER(ctypes.c_double)), ("precision", ctypes.c_int),
                ("filter", ctypes.c_int), ("reg", ctypes.POINTER(ctypes.c_double)),
                ("nreg", ctypes.c_int)]


class _SmDesc(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int), ("width", ctypes.c_int), ("ksize", ctypes.c_int),
                ("nlevels", ctypes.c_int), ("weights", ctypes.POINTER(ctypes.c_double)),
                ("nweights", ctypes.c_size_t), ("arch", ctypes.c_int), ("modes", ctypes.c_int),
                ("level_layers", ctypes.POINTER(ctypes.c_int))]

SMOOTHER_CNN, SMOOTHER_FNO = 0, 1


class SolveInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("status", ctypes.c_int), ("relres", ctypes.c_double)]


class _SolveItem(ctypes.Structure):
    _fields_ = [("hier", ctypes.c_void_p), ("batch", ctypes.c_int), ("f", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("info", ctypes.POINTER(SolveInfo))]


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load libnmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_2603_01064_gb300/build.py "
                           "(or __graft_entry__.build()); there is no fallback path")
    L = ctypes.CDLL(_LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    sig = {
        "nmg_create": (I, [ctypes.POINTER(P), I, P]),
        "nmg_destroy": (V, [P]),
        "nmg_setup": (I, [P, ctypes.POINTER(_OpDesc), ctypes.POINTER(_SmDesc), ctypes.POINTER(P)]),
        "nmg_destroy_hier": (V, [P]),
        "nmg_solve": (I, [P, P, I, P, P, D, I, ctypes.POINTER(SolveInfo)]),
        "nmg_solve_host": (I, [P, P, I, P, P, D, I, ctypes.POINTER(SolveInfo)]),
        "nmg_solve_host_zero": (I, [P, P, I, P, P, D, I, ctypes.POINTER(SolveInfo)]),
        "nmg_solve_multi": (I, [P, I, ctypes.POINTER(_SolveItem), D, I]),
        "nmg_solve_mg_jacobi": (I, [P, P, I, P, P, D, I, I, I, ctypes.POINTER(SolveInfo)]),
        "nmg_solve_cg": (I, [P, P, I, P, P, D, I, ctypes.POINTER(SolveInfo)]),
        "nmg_server_create": (I, [P, ctypes.c_size_t, D, I, ctypes.POINTER(P)]),
        "nmg_server_destroy": (V, [P]),
        "nmg_server_add_operator": (I, [P, P, I, ctypes.POINTER(I)]),
        "nmg_server_submit": (I, [P, I, P, P, ctypes.POINTER(ctypes.c_longlong)]),
        "nmg_server_step": (I, [P, ctypes.POINTER(I)]),
        "nmg_server_query": (I, [P, ctypes.c_longlong, ctypes.POINTER(SolveInfo), ctypes.POINTER(I),
                                 ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "nmg_server_stats": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_size_t)]),
        "nmg_cycle": (I, [P, P, I, P, P]),
        "nmg_residual": (I, [P, P, I, I, P, P, P, ctypes.POINTER(D)]),
        "nmg_residual_restrict": (I, [P, P, I, I, P, P, P]),
        "nmg_residual_noalloc": (I, [P, P, I, I, P, P, P, ctypes.POINTER(D)]),
        "nmg_smooth": (I, [P, P, I, I, P, P]),
        "nmg_filter_update": (I, [P, P, I, I, P, P, P]),
        "nmg_coarse_solve": (I, [P, P, I, P, P]),
        "nmg_prolong_correct": (I, [P, P, I, I, P, P]),
        "nmg_hier_info": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                              ctypes.POINTER(I)]),
        "nmg_hier_level_dense": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "nmg_host_level_dense": (I, [ctypes.POINTER(_OpDesc), I, ctypes.POINTER(I), ctypes.POINTER(I),
                                     ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "nmg_launch_count": (ctypes.c_longlong, [P]),
        "nmg_profile_enable": (I, [P, I]),
        "nmg_set_graphs": (I, [P, I]),
        "nmg_set_wait_limit": (I, [P, ctypes.c_longlong]),
        "nmg_inject_stall": (I, [P, I]),
        "nmg_autotune": (I, [P, P, I, ctypes.c_char_p]),
        "nmg_hier_tuning": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                ctypes.POINTER(I)]),
        "nmg_profile_read": (I, [P, I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D),
                                 ctypes.POINTER(D)]),
        "nmg_sync": (I, [P]),
        "nmg_status_str": (ctypes.c_char_p, [I]),
        "nmg_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(t):
    """Device pointer of a contiguous torch tensor (or None)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def host_level_dense(*, dim: int, n: int, levels: int, alpha: float, taps, level: int,
                     reg=None):
    """The Galerkin hierarchy built on the host by the library (no GPU):
    level `level`'s factors in dense form, (K_l, M_l) in 2D or A_l in 1D,
    exactly as a hierarchy set up from the same description holds them."""
    L = lib()
    t = np.ascontiguousarray(taps, dtype=np.float64)
    r = None
    if reg is not None:
        r = np.ascontiguousarray(np.concatenate([np.asarray(reg[0], np.float64),
                                                 np.asarray(reg[1], np.float64)]))
    dp = ctypes.POINTER(ctypes.c_double)
    op = _OpDesc(dim, n, levels, alpha, len(t), t.ctypes.data_as(dp), PRECISIONS["fp64"], 1,
                 r.ctypes.data_as(dp) if r is not None else None, 0 if r is None else r.size)
    nl, wk, wm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = L.nmg_host_level_dense(ctypes.byref(op), level, ctypes.byref(nl), ctypes.byref(wk),
                                ctypes.byref(wm), None, None)
    if rc != 0:
        raise NMGError(rc, L.nmg_status_str(rc).decode())
    m = nl.value
    K = np.zeros((m, m))
    M = np.zeros((m, m)) if dim == 2 else None
    rc = L.nmg_host_level_dense(ctypes.byref(op), level, None, None, None, K.ctypes.data_as(dp),
                                M.ctypes.data_as(dp) if M is not None else None)
    if rc != 0:
        raise NMGError(rc, L.nmg_status_str(rc).decode())
    return (K, M) if dim == 2 else K


def pack_weights(levels: Sequence[Sequence[tuple]]) -> np.ndarray:
    """Flatten [[(W, b), ...] per level] into the ABI order (per level, per
    layer: W in PyTorch Conv layout, then b)."""
    parts = []
    for lv in levels:
        for W, b in lv:
            parts.append(np.asarray(W, np.float64).ravel())
            parts.append(np.asarray(b, np.float64).ravel())
    return np.ascontiguousarray(np.concatenate(parts)) if parts else np.zeros(0)


def pack_fno_weights(levels) -> np.ndarray:
    """Flatten per-level FNO weights dict(lift=(W, b), layers=[(W, b, R)],
    proj=(W, b)) into the ABI order: lift W, b; per layer W (PyTorch Conv2d
    layout), b, Re R, Im R (R as [2][in][out][m][m]); projection W, b."""
    parts = []
    for lv in levels:
        parts += [np.asarray(a, np.float64).ravel() for a in lv["lift"]]
        for W, b, R in lv["layers"]:
            R = np.asarray(R, np.complex128)
            parts += [np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64).ravel(),
                      R.real.ravel(), R.imag.ravel()]
        parts += [np.asarray(a, np.float64).ravel() for a in lv["proj"]]
    return np.ascontiguousarray(np.concatenate(parts))


def load_weights(path: str):
    """Read a trained smoother file: CNN (npz: l{level}_w{layer},
    l{level}_b{layer}) or FNO (meta_arch = "fno": per level a dict of lift,
    layers (W, b, R) and proj, see pack_fno_weights)."""
    z = np.load(path)
    nl = int(z["meta_smoother_levels"])
    if "meta_arch" in z.files and str(z["meta_arch"]) == "fno":
        nk = len([k for k in z.files if k.startswith("l0_k") and k.endswith("_w")])
        return [dict(lift=(z[f"l{l}_lift_w"], z[f"l{l}_lift_b"]),
                     layers=[(z[f"l{l}_k{i}_w"], z[f"l{l}_k{i}_b"],
                              z[f"l{l}_k{i}_rre"] + 1j * z[f"l{l}_k{i}_rim"]) for i in range(nk)],
                     proj=(z[f"l{l}_proj_w"], z[f"l{l}_proj_b"])) for l in range(nl)]
    depth = [len([k for k in z.files if k.startswith(f"l{l}_w")]) for l in range(nl)]
    return [[(z[f"l{l}_w{i}"], z[f"l{l}_b{i}"]) for i in range(depth[l])] for l in range(nl)]


class Context:
    """A CUDA device + stream for the library."""

    def __init__(self, device: int = 0, stream=None):
        L = lib()
        self._h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(int(stream))
        rc = L.nmg_create(ctypes.byref(self._h), int(device), s)
        if rc != 0:
            raise NMGError(rc, L.nmg_status_str(rc).decode())
        self.device = device
        self.graphs = True

    def check(self, rc):
        if rc != 0:
            L = lib()
            raise NMGError(rc, f"{L.nmg_status_str(rc).decode()}: {L.nmg_last_error(self._h).decode()}")

    def sync(self):
        self.check(lib().nmg_sync(self._h))

    def launches(self) -> int:
        return int(lib().nmg_launch_count(self._h))

    def set_graphs(self, enable: bool):
        """Replay captured CUDA graphs per outer iteration (default) or launch eagerly."""
        self.check(lib().nmg_set_graphs(self._h, 1 if enable else 0))
        self.graphs = bool(enable)

    def set_wait_limit(self, ns: int):
        """Bound of every device wait of the tensor-core kernels, in ns."""
        self.check(lib().nmg_set_wait_limit(self._h, int(ns)))

    def inject_stall(self, enable: bool):
        """Test hook: tensor-core smoother launches give up on a wait that
        nothing ends (after the wait limit), reporting NMG_ERR_TIMEOUT."""
        self.check(lib().nmg_inject_stall(self._h, 1 if enable else 0))

    def profile(self, enable: bool):
        self.check(lib().nmg_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self, kind: int):
        """(launches, total device ms, work units) recorded for a kernel class."""
        c = ctypes.c_longlong()
        ms = ctypes.c_double()
        u = ctypes.c_double()
        self.check(lib().nmg_profile_read(self._h, kind, ctypes.byref(c), ctypes.byref(ms),
                                          ctypes.byref(u)))
        return c.value, ms.value, u.value

    def close(self):
        if self._h:
            lib().nmg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """One operator's level hierarchy (nmg_setup)."""

    def __init__(self, ctx: Context, *, dim: int, n: int, levels: int, alpha: float,
                 taps, precision="fp32", filter: bool = True, weights=None,
                 layers=None, width=None, ksize=None, reg=None):
        """reg: None (D = I) or (diag, off) of the tridiagonal regularisation
        matrix D of the anisotropic 1D case (A = alpha D + K)."""
        L = lib()
        self.ctx = ctx
        self.dim, self.n, self.levels, self.alpha = dim, n, levels, alpha
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._taps = np.ascontiguousarray(taps, dtype=np.float64)
        self._reg = None
        if reg is not None:
            self._reg = np.ascontiguousarray(np.concatenate([np.asarray(reg[0], np.float64),
                                                             np.asarray(reg[1], np.float64)]))
        op = _OpDesc(dim, n, levels, alpha, len(self._taps),
                     self._taps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     self.precision, 1 if filter else 0,
                     self._reg.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                     if self._reg is not None else None,
                     0 if self._reg is None else self._reg.size)
        smp = None
        if weights is not None and isinstance(weights[0], dict):
            # FNO smoother (Appendix A): dims from the first level's arrays
            lv0 = weights[0]
            W1, _, R1 = lv0["layers"][0]
            layers, width, ksize = len(lv0["layers"]), np.asarray(W1).shape[0], np.asarray(W1).shape[-1]
            self._w = pack_fno_weights(weights)
            sm = _SmDesc(layers, width, ksize, len(weights),
                         self._w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self._w.size,
                         SMOOTHER_FNO, np.asarray(R1).shape[-1])
            smp = ctypes.byref(sm)
        elif weights is not None:
            if layers is None:
                W0 = np.asarray(weights[0][0][0])  # first layer: [width, 1, k(, k)]
                layers, width, ksize = len(weights[0]), W0.shape[0], W0.shape[-1]
            self._w = pack_weights(weights)
            # per-level depths (levels may differ, Appendix A's Table 6)
            self._depths = np.array([len(lv) for lv in weights], dtype=np.int32)
            sm = _SmDesc(layers, width, ksize, len(weights),
                         self._w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self._w.size,
                         SMOOTHER_CNN, 0, self._depths.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
            smp = ctypes.byref(sm)
        self._h = ctypes.c_void_p()
        ctx.check(L.nmg_setup(ctx._h, ctypes.byref(op), smp, ctypes.byref(self._h)))

    # ---- shapes / dtypes
    def size(self, level: int = 0) -> int:
        return self.n >> level

    def shape(self, batch: int, level: int = 0):
        m = self.size(level)
        return (batch, m) if self.dim == 1 else (batch, m, m)

    # ---- solves
    def solve(self, f, u, rtol=1e-6, max_cycles=100):
        """Device solve; f, u torch CUDA tensors of the hierarchy's types.
        Returns (cycles, status, relres) numpy arrays."""
        B = f.shape[0]
        info = (SolveInfo * max(B, 1))()
        self.ctx.check(lib().nmg_solve(self.ctx._h, self._h, B, _ptr(f), _ptr(u), float(rtol),
                                       int(max_cycles), info))
        return _unpack(info, B)

    def solve_mg_jacobi(self, f, u, rtol=1e-6, max_cycles=5000, nu1=5, nu2=0):
        """Classical comparator: V-cycles of Algorithm 1 with weighted Jacobi
        smoothing (nu1 pre-, nu2 post-smoothing steps).  Returns (cycles,
        status, relres)."""
        B = f.shape[0]
        info = (SolveInfo * max(B, 1))()
        self.ctx.check(lib().nmg_solve_mg_jacobi(self.ctx._h, self._h, B, _ptr(f), _ptr(u),
                                                 float(rtol), int(max_cycles), int(nu1), int(nu2),
                                                 info))
        return _unpack(info, B)

    def solve_cg(self, f, u, rtol=1e-6, max_iters=10000):
        """Classical comparator: conjugate gradients.  Returns (iterations,
        status, relres)."""
        B = f.shape[0]
        info = (SolveInfo * max(B, 1))()
        self.ctx.check(lib().nmg_solve_cg(self.ctx._h, self._h, B, _ptr(f), _ptr(u), float(rtol),
                                          int(max_iters), info))
        return _unpack(info, B)

    def solve_host(self, f: np.ndarray, u: np.ndarray, rtol=1e-6, max_cycles=100,
                   zero_start: bool = False):
        """Solve from host (numpy) buffers; u is updated in place.  With
        zero_start the solve starts from u = 0 and u is output only (not
        read or copied to the device)."""
        assert f.flags.c_contiguous and u.flags.c_contiguous
        B = f.shape[0]
        info = (SolveInfo * max(B, 1))()
        fn = lib().nmg_solve_host_zero if zero_start else lib().nmg_solve_host
        self.ctx.check(fn(self.ctx._h, self._h, B, ctypes.c_void_p(f.ctypes.data),
                          ctypes.c_void_p(u.ctypes.data), float(rtol), int(max_cycles), info))
        return _unpack(info, B)

    def cycle(self, f, u):
        self.ctx.check(lib().nmg_cycle(self.ctx._h, self._h, f.shape[0], _ptr(f), _ptr(u)))

    # ---- single steps
    def residual(self, level, x, y, r, norms=False):
        B = x.shape[0]
        out = (ctypes.c_double * max(B, 1))() if norms else None
        self.ctx.check(lib().nmg_residual(self.ctx._h, self._h, level, B, _ptr(x), _ptr(y),
                                          _ptr(r), out))
        return np.array(out[:B]) if norms else None

    def residual_noalloc(self, level, x, y, r, norms=False):
        """nmg_residual with its scratch in the library's fixed array: no
        device allocation (limit NOALLOC_SCRATCH_BYTES; calls that overlap
        on the device race on the shared array)."""
        B = x.shape[0]
        out = (ctypes.c_double * max(B, 1))() if norms else None
        self.ctx.check(lib().nmg_residual_noalloc(self.ctx._h, self._h, level, B, _ptr(x),
                                                  _ptr(y), _ptr(r), out))
        return np.array(out[:B]) if norms else None

    def residual_restrict(self, level, x, y, yc):
        self.ctx.check(lib().nmg_residual_restrict(self.ctx._h, self._h, level, x.shape[0],
                                                   _ptr(x), _ptr(y), _ptr(yc)))

    def smooth(self, level, b, h):
        self.ctx.check(lib().nmg_smooth(self.ctx._h, self._h, level, b.shape[0], _ptr(b), _ptr(h)))

    def filter_update(self, level, xstar, h, x):
        self.ctx.check(lib().nmg_filter_update(self.ctx._h, self._h, level, h.shape[0],
                                               _ptr(xstar), _ptr(h), _ptr(x)))

    def coarse_solve(self, y, x):
        self.ctx.check(lib().nmg_coarse_solve(self.ctx._h, self._h, y.shape[0], _ptr(y), _ptr(x)))

    def prolong_correct(self, level, e, x):
        self.ctx.check(lib().nmg_prolong_correct(self.ctx._h, self._h, level, x.shape[0],
                                                 _ptr(e), _ptr(x)))

    def autotune(self, batch: int, cache_path: str | None = None):
        """Time the candidate launch shapes per level and keep the fastest."""
        self.ctx.check(lib().nmg_autotune(self.ctx._h, self._h, int(batch),
                                          cache_path.encode() if cache_path else None))

    def tuning(self, level: int):
        v = [ctypes.c_int() for _ in range(4)]
        self.ctx.check(lib().nmg_hier_tuning(self._h, level, *[ctypes.byref(x) for x in v]))
        return dict(zip(["res_tile", "rst_tile", "ref_tile", "filt_mode"], [x.value for x in v]))

    # ---- inspection
    def level_dense(self, level):
        m = self.size(level)
        K = np.zeros((m, m))
        M = np.zeros((m, m))
        dp = ctypes.POINTER(ctypes.c_double)
        rc = lib().nmg_hier_level_dense(self._h, level, K.ctypes.data_as(dp), M.ctypes.data_as(dp))
        self.ctx.check(rc)
        return (K, M) if self.dim == 2 else K

    def close(self):
        # a hierarchy finalised after its context (interpreter shutdown) is
        # left to the process exit: its context's device state is gone
        if self._h and self.ctx._h:
            lib().nmg_destroy_hier(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_multi(ctx: "Context", items, rtol=1e-6, max_cycles=100):
    """Solve several (hierarchy, f, u) batches together (nmg_solve_multi).
    items: list of (Hierarchy, f, u) with torch CUDA tensors; returns a list of
    (cycles, status, relres) per item."""
    arr = (_SolveItem * max(len(items), 1))()
    infos = []
    for i, (G, f, u) in enumerate(items):
        B = f.shape[0]
        inf = (SolveInfo * max(B, 1))()
        infos.append((inf, B))
        arr[i] = _SolveItem(G._h.value, B, _ptr(f).value if B else None,
                            _ptr(u).value if B else None, inf)
    ctx.check(lib().nmg_solve_multi(ctx._h, len(items), arr, float(rtol), int(max_cycles)))
    return [_unpack(inf, B) for inf, B in infos]


class Server:
    """Continuous-batching solve server (nmg_server_*): resident hierarchies,
    per-operator slot pools, one outer iteration per live request per step."""

    def __init__(self, ctx: "Context", budget_bytes: int, rtol=1e-6, max_cycles=100):
        self.ctx = ctx
        self._h = ctypes.c_void_p()
        ctx.check(lib().nmg_server_create(ctx._h, int(budget_bytes), float(rtol), int(max_cycles),
                                          ctypes.byref(self._h)))
        self._keep = {}

    def add_operator(self, G: "Hierarchy", slots: int) -> int:
        op = ctypes.c_int()
        self.ctx.check(lib().nmg_server_add_operator(self._h, G._h, int(slots), ctypes.byref(op)))
        return op.value

    def submit(self, op: int, f: np.ndarray, u_out: np.ndarray) -> int:
        """f, u_out: contiguous host arrays of the operator's f and u types;
        u_out must stay alive until the request is done."""
        assert f.flags.c_contiguous and u_out.flags.c_contiguous
        rid = ctypes.c_longlong()
        self.ctx.check(lib().nmg_server_submit(self._h, int(op), ctypes.c_void_p(f.ctypes.data),
                                               ctypes.c_void_p(u_out.ctypes.data),
                                               ctypes.byref(rid)))
        self._keep[rid.value] = u_out
        return rid.value

    def step(self) -> int:
        c = ctypes.c_int()
        self.ctx.check(lib().nmg_server_step(self._h, ctypes.byref(c)))
        return c.value

    def query(self, rid: int):
        """(state, (cycles, status, relres), t_submit, t_admit, t_done)."""
        info = SolveInfo()
        st = ctypes.c_int()
        t = [ctypes.c_double() for _ in range(3)]
        self.ctx.check(lib().nmg_server_query(self._h, int(rid), ctypes.byref(info), ctypes.byref(st),
                                              *[ctypes.byref(x) for x in t]))
        if st.value == 2:
            self._keep.pop(rid, None)
        return st.value, (info.cycles, info.status, info.relres), t[0].value, t[1].value, t[2].value

    def stats(self):
        q, r = ctypes.c_int(), ctypes.c_int()
        b = ctypes.c_size_t()
        self.ctx.check(lib().nmg_server_stats(self._h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)))
        return q.value, r.value, b.value

    def close(self):
        if self._h and self.ctx._h:
            lib().nmg_server_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _unpack(info, B):
    cyc = np.array([info[i].cycles for i in range(B)], dtype=np.int64)
    st = np.array([info[i].status for i in range(B)], dtype=np.int64)
    rr = np.array([info[i].relres for i in range(B)], dtype=np.float64)
    return cyc, st, rr
