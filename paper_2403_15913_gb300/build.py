"""Builds the CUDA library libkkt_gb300.so in-tree for sm_103a with nvcc.

The translation units are compiled in parallel and linked against the shared
CUDA runtime (the one PyTorch also loads), so CUDA streams created by torch
are valid handles inside the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libkkt_gb300.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)
# the bounds-check build (-DKKT_BOUNDS_CHECK=1): same C ABI, every map index
# tested on the device; used by the tests, never by the product path
LIB_PATH_CHECKED = os.path.join(HERE, "libkkt_gb300_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kkt.cu", "tray.cu", "ipm.cu", "serve.cu", "symbolic.cpp"]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the KKT library")


def build(verbose: bool = False, debug_checks: bool = False) -> str:
    """Compile every source and link the shared library; returns its path
    (debug_checks: the bounds-check build, a separate library)."""
    nvcc = _nvcc()
    obj_dir = os.path.join(HERE, "_build_checked" if debug_checks else "_build")
    lib_path = LIB_PATH_CHECKED if debug_checks else LIB_PATH
    os.makedirs(obj_dir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-Xcompiler", "-fPIC,-O2",
              "-lineinfo"] + ARCH
    if debug_checks:
        common += ["-DKKT_BOUNDS_CHECK=1"]
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(obj_dir, src.replace(".", "_") + ".o")
        objs.append(obj)
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "cu"] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out.decode(errors='replace')}")
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib_path + ".tmp"
    cmd = [nvcc, "-shared", "-cudart", "shared"] + ARCH + objs + ["-lpthread", "-o", tmp]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True))
