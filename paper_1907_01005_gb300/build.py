"""Builds libfe_mf.so in the package directory with nvcc for sm_103a.

Each translation unit is compiled in its own nvcc process (in parallel),
then the objects are linked into one shared library.  Usage:
    python -m paper_1907_01005_gb300.build [--verbose] [--debug]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libfe_mf.so")
SOURCES = ["host.cpp", "apply.cu", "apply_unit.cu", "apply_cellmat.cu", "gram.cu", "gram_tc.cu", "mmult.cu", "mmult_tc.cu", "peak.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfe_mf.so")


def flags(debug: bool = False, ptxas_verbose: bool = False) -> list[str]:
    f = ["-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O3",
         "-I" + os.path.join(PKG, "..", "include")]
    if debug:
        f.append("-DFE_DEBUG_BOUNDS=1")
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f


def _compile(src: str, obj: str, fl: list[str]) -> tuple[str, str]:
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + fl
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return src, r.stdout + r.stderr


def build(verbose: bool = False, debug: bool = False, ptxas_verbose: bool = False, out: str = LIB) -> str:
    bdir = os.path.join(PKG, "_build")
    os.makedirs(bdir, exist_ok=True)
    fl = flags(debug, ptxas_verbose)
    objs = [os.path.join(bdir, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for src, log in ex.map(lambda so: _compile(so[0], so[1], fl), zip(SOURCES, objs)):
            if verbose and log.strip():
                print(f"[{src}]\n{log}", file=sys.stderr)
    tmp = out + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + [ARCH, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    build(verbose="--verbose" in sys.argv, debug="--debug" in sys.argv,
          ptxas_verbose="--ptxas" in sys.argv)
    print(LIB)
