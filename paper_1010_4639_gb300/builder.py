"""Builds ``libgbcg.so`` in-tree for sm_103a (GB300).

Six translation units compiled in parallel: ``csrc/gbcg.cu`` (kernels and
the C ABI, nvcc), ``csrc/static_solve.cu`` (the allocation-free solve, nvcc),
``csrc/batch.cu`` (the batched multi-right-hand-side solver, nvcc),
``csrc/grad.cu`` (gradient kernels of the differentiable solve, nvcc),
``csrc/ablation.cu`` (the paper's 2010 solver structure, a measurement
baseline, nvcc) and ``csrc/layout.cpp`` (host-side layout construction,
g++), linked by nvcc into a shared library next to this file.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgbcg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = [os.path.join(CSRC, f) for f in ("gbcg.cu", "static_solve.cu", "batch.cu", "grad.cu", "ablation.cu", "layout.cpp",
                                              "kernels.cuh", "layout.h")]
HEADERS = [os.path.join(INCLUDE, "gbcg.h")]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in SOURCES + HEADERS + [__file__])


def build(verbose: bool = False, force: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cu_obj = os.path.join(BUILD, "gbcg.o")
    st_obj = os.path.join(BUILD, "static_solve.o")
    bt_obj = os.path.join(BUILD, "batch.o")
    gr_obj = os.path.join(BUILD, "grad.o")
    ab_obj = os.path.join(BUILD, "ablation.o")
    cpp_obj = os.path.join(BUILD, "layout.o")
    cmds = [
        [nvcc, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
         "-I", INCLUDE, os.path.join(CSRC, "gbcg.cu"), "-o", cu_obj],
        [nvcc, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
         "-I", INCLUDE, os.path.join(CSRC, "static_solve.cu"), "-o", st_obj],
        [nvcc, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
         "-I", INCLUDE, os.path.join(CSRC, "batch.cu"), "-o", bt_obj],
        [nvcc, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
         "-I", INCLUDE, os.path.join(CSRC, "grad.cu"), "-o", gr_obj],
        [nvcc, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
         "-I", INCLUDE, os.path.join(CSRC, "ablation.cu"), "-o", ab_obj],
        ["g++", "-c", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE,
         os.path.join(CSRC, "layout.cpp"), "-o", cpp_obj],
    ]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    errors = []
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose and out:
            print(out, file=sys.stderr)
        if p.returncode != 0:
            errors.append(f"{' '.join(c)}\n{out}")
    if errors:
        raise RuntimeError("building libgbcg.so failed:\n" + "\n".join(errors))
    tmp = LIB + ".tmp"
    subprocess.run([nvcc, "-shared", *ARCH, cu_obj, st_obj, bt_obj, gr_obj, ab_obj, cpp_obj, "-o", tmp], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
