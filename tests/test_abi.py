"""The C-ABI library loads without a GPU and exports every function that
include/nmg.h declares; host-side argument handling of the binding."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nmg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2603_01064_gb300 as nmg
    from paper_2603_01064_gb300 import build
    if not os.path.exists(nmg.lib_path()):
        build.build()
    return nmg.lib_path()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["nmg_create", "nmg_setup", "nmg_solve", "nmg_solve_host", "nmg_cycle",
                 "nmg_destroy", "nmg_destroy_hier", "nmg_status_str", "nmg_residual",
                 "nmg_residual_restrict", "nmg_smooth", "nmg_filter_update", "nmg_coarse_solve",
                 "nmg_prolong_correct"]:
        assert must in names


def test_noalloc_limit_matches_header():
    """The binding's copy of NMG_NOALLOC_SCRATCH_BYTES equals the header's."""
    import paper_2603_01064_gb300 as nmg
    src = open(os.path.join(ROOT, "include", "nmg.h")).read()
    m = re.search(r"#define\s+NMG_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", src)
    assert m, "define not found"
    assert int(m.group(1)) << int(m.group(2)) == nmg.NOALLOC_SCRATCH_BYTES


def test_precision_constants_match_header():
    """The binding's precision numbers equal the header's nmg_precision."""
    import paper_2603_01064_gb300 as nmg
    src = open(os.path.join(ROOT, "include", "nmg.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} nmg_precision;", src).group(1)
    hdr = {k: int(v) for k, v in re.findall(r"NMG_([A-Z0-9_]+)\s*=\s*(\d+)", body)}
    assert hdr and set(hdr) == {k.upper() for k in nmg.PRECISIONS}
    for name, val in nmg.PRECISIONS.items():
        assert hdr[name.upper()] == val, name


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    import paper_2603_01064_gb300 as nmg
    L = nmg.lib()
    assert L.nmg_status_str(0) == b"ok"
    assert L.nmg_status_str(-3).startswith(b"coarsest")
    assert L.nmg_status_str(-99) == b"unknown status"


def test_create_rejects_bad_device_without_gpu(libpath):
    import paper_2603_01064_gb300 as nmg
    h = ctypes.c_void_p()
    assert nmg.lib().nmg_create(ctypes.byref(h), 12345, None) == -1


def test_pack_weights_order():
    import nmg_inputs as I
    import paper_2603_01064_gb300 as nmg
    W = I.random_cnn_weights(2, 2, seed=1)
    p = nmg.pack_weights(W)
    assert p.size == 2 * 19105
    assert p[0] == W[0][0][0].ravel()[0]
    assert p[288] == W[0][0][1][0]          # bias after the first conv weights
    assert p[19105] == W[1][0][0].ravel()[0]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback path: without the built library every entry raises."""
    import paper_2603_01064_gb300 as nmg
    monkeypatch.setattr(nmg, "_lib", None)
    monkeypatch.setattr(nmg, "_LIB_PATH", str(tmp_path / "libnmg.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        nmg.lib()
    with pytest.raises(RuntimeError, match="no fallback"):
        nmg.Context(0)
    with pytest.raises(RuntimeError, match="no fallback"):
        nmg.host_level_dense(dim=2, n=16, levels=2, alpha=1e-2, taps=[1.0], level=0)
