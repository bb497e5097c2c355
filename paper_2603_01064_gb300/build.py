"""Compile the CUDA library libnmg.so in-tree for sm_103a (GB300).

Each translation unit is compiled in parallel with nvcc, then linked into a
shared library next to this file (`_build/libnmg.so`).  Called by
``__graft_entry__.build()`` and by the binding when the library is missing
is an error, not a trigger: the binding never compiles implicitly.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libnmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "hierarchy.cpp", "k_ops.cu", "k_cnn.cu", "k_cnn_bf16.cu", "k_filter.cu",
           "k_coarse.cu", "k_refine.cu", "k_stencil_f32.cu", "k_stencil_f64.cu", "k_fno.cu", "k_wide.cu", "k_classic.cu"]


def _nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    for c in ("/usr/local/cuda/bin/nvcc",):
        if os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra_ptxas=False):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(HERE, "..", "include")] + ARCH
    if extra_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    cmds = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        lang = ["-x", "cu"] if src.endswith(".cu") else []
        cmds.append([nvcc, *_flags(ptxas_info), *lang, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        for cmd, r in ex.map(run, cmds):
            if verbose or ptxas_info or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    link = [nvcc, "-shared", *ARCH, "-o", LIB, *objs, "-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv))
