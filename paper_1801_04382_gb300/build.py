"""Build the CUDA library ``libkrotov_traj.so`` in-tree for sm_103a.

nvcc compiles every kernel translation unit (``csrc/*.cu``) and g++ the host runtime
(``csrc/*.cpp``), all in parallel; the objects are linked into one shared library against
the CUDA runtime.  The output goes to ``paper_1801_04382_gb300/_lib/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB_NAME = "libkrotov_traj.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def lib_path() -> str:
    return os.path.join(OUT_DIR, LIB_NAME)


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    return res.stdout + res.stderr


def build(verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile and link the library; returns its path."""
    cuda = cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = os.path.join(cuda, "include")
    libdir = next(p for p in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"),
                              os.path.join(cuda, "targets", "sbsa-linux", "lib"),
                              os.path.join(cuda, "targets", "x86_64-linux", "lib")) if os.path.isdir(p))
    os.makedirs(OUT_DIR, exist_ok=True)
    cmds, objs = [], []
    for src in sorted(os.listdir(CSRC)):
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", path, "-o", obj]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
        elif src.endswith(".cpp"):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-I" + inc, "-c", path, "-o", obj]
        else:
            continue
        cmds.append(cmd)
        objs.append(obj)
    with cf.ThreadPoolExecutor(len(cmds)) as ex:
        outs = list(ex.map(lambda c: _run(c, verbose), cmds))
    if ptxas_verbose:
        print("\n".join(outs))
    tmp = lib_path() + ".tmp"
    _run([nvcc, *ARCH, "-shared", *objs, "-o", tmp, "-L" + libdir, "-lcudart"], verbose)
    os.replace(tmp, lib_path())
    return lib_path()


if __name__ == "__main__":
    print(build(verbose=True, ptxas_verbose="-v" in sys.argv))
