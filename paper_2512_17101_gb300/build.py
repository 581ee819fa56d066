"""Builds libdg.so in-tree (nvcc for sm_103a; the host C++ with g++).

Translation units are compiled in parallel into ``_build/`` and linked into
``paper_2512_17101_gb300/libdg.so``.  No cmake, no torch extension machinery.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libdg.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    hs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    hs.append(os.path.join(INCLUDE, "dg.h"))
    return hs


def _digest(cmd, path):
    """Hash of the compile command, the source and every header: an object is reused only when all
    of them are byte-identical to the ones it was built from (timestamps are not trusted: a copied
    tree keeps stale objects newer than their sources)."""
    h = hashlib.sha256(" ".join(cmd).encode())
    for f in [path] + _headers():
        with open(f, "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()


def _compile(src, verbose=False, ptxas_info=False):
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    if src.endswith(".cu"):
        cmd = [NVCC, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
               "-c", path, "-o", obj]
        if ptxas_info:
            cmd[1:1] = ["-Xptxas", "-v"]
    else:
        cmd = ["g++", "-O2", "-fPIC", "-std=c++17", "-I", INCLUDE, "-I", CSRC, "-I",
               os.path.join(CUDA_HOME, "include"), "-c", path, "-o", obj]
    stamp = obj + ".sha256"
    key = _digest(cmd, path) + " " + os.uname().machine
    if not ptxas_info and os.path.exists(obj) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == key:
                return obj, ""
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    with open(stamp, "w") as fh:
        fh.write(key + "\n")
    return obj, (r.stdout + r.stderr) if (verbose or ptxas_info) else ""


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link libdg.so; returns its path."""
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, ptxas_info), srcs))
    objs = [o for o, _ in results]
    if verbose or ptxas_info:
        for (_, log), s in zip(results, srcs):
            if log:
                print(f"--- {s}\n{log}")
    tmp = LIB + ".tmp"
    cmd = [NVCC, ARCH, "-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking libdg.so failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    shutil.move(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv))
