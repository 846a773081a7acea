"""Build the CUDA library libicmpt.so in-tree, for sm_103a only.

The translation units are compiled in parallel with nvcc and linked into
``paper_1501_05630_gb300/_build/libicmpt.so`` (the CUDA runtime is linked
statically, so the library depends only on the driver).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libicmpt.so")
SOURCES = ["pt_icm.cu", "fused_pmj.cu", "fused_gauss.cu", "cluster_icm.cu", "icm_api.cpp", "icm_server.cpp",
           "icm_static.cu", "percolation.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
         "-I", CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


# Checked build: every guarded index of the fused kernel is tested against its
# bound and an out-of-range index is recorded (icm_debug_check) and replaced by
# 0, so that the access stays in bounds.  Built apart, never on the product path.
CHECKED_BUILD = os.path.join(PKG, "_build_checked")
CHECKED_LIB = os.path.join(CHECKED_BUILD, "libicmpt.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "icmpt.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    out_dir, lib = (CHECKED_BUILD, CHECKED_LIB) if checked else (BUILD, LIB)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    cmds = []
    defs = ["-DICM_CHECKED"] if checked else []
    for src in SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        objs.append(obj)
        extra = ["-x", "cu"] if src.endswith(".cu") else []
        cmds.append([nvcc, *ARCH, *FLAGS, *defs, *extra, "-c", os.path.join(CSRC, src), "-o", obj])
    if verbose:
        cmds[0].insert(1, "-Xptxas=-v")
    with cf.ThreadPoolExecutor(len(cmds)) as ex:
        for r in ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds):
            if r.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
            if verbose and r.stderr:
                print(r.stderr)
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
