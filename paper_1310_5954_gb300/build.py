"""Build libletkf.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked against the CUDA runtime
only (every kernel is the library's own).  The library is written next to this file
(lib/libletkf.so) and is git-ignored.
"""

from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libletkf.so")
SOURCES = ["host.cpp", "plain.cu", "misc.cu", "fused.cu", "noise.cu", "piston.cu", "gemm.cu", "global.cu", "server.cpp", "tune.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libletkf")


def _compile(nvcc: str, src: str, obj: str, verbose: bool) -> None:
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
           os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd[5:5] = ["--expt-relaxed-constexpr"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 or verbose:
        sys.stderr.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}")


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every source and link lib/libletkf.so; returns the library path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    objdir = os.path.join(OUT_DIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    inc = os.path.join(HERE, "..", "include")
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(inc, f) for f in os.listdir(inc)]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest and not verbose:
        return LIB
    nvcc = _nvcc()
    objs = [os.path.join(objdir, s + ".o") for s in SOURCES]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        futs = [ex.submit(_compile, nvcc, s, o, verbose) for s, o in zip(SOURCES, objs)]
        for f in futs:
            f.result()
    cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link of libletkf.so failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
