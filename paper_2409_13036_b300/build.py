"""Build librafem.so in-tree for sm_103a (B300) with nvcc.

Usage: python -m paper_2409_13036_b300.build [--verbose]
The library is written next to this file, so it travels with the source tree, together with the SHA-256 of
the sources it was built from (librafem.so.sha256): a library whose sources changed is rebuilt.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import concurrent.futures as cf
import hashlib

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "librafem.so")
HASH = LIB + ".sha256"  # source hash of the build that produced LIB
OBJDIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp,-O2", "-I" + INCLUDE,
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
SOURCES = ["api.cu", "adjoint.cu", "assembly.cu", "assembly_dw.cu", "bicgstab.cu", "bicgstab_ring.cu", "gmres.cu", "ilu.cu", "ilu_ring.cu", "krylov.cu", "mono_fgmres.cu", "coupled_gather.cu", "noalloc.cu", "project.cu", "setup.cpp"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
        print(" ".join(cmd))
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout, r.stderr)
    return obj


def source_hash() -> str:
    """SHA-256 over every input of the build: the sources, the headers, this script (flags included) and the nvcc
    version. A library whose recorded hash differs (or is missing) is rebuilt, whatever the file times say."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    hdrs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    hdrs.append(os.path.join(INCLUDE, "rafem.h"))
    h = hashlib.sha256()
    for p in srcs + hdrs + [os.path.abspath(__file__)]:
        h.update(os.path.basename(p).encode() + b"\0")
        with open(p, "rb") as f:
            h.update(f.read())
    r = subprocess.run([nvcc(), "--version"], capture_output=True, text=True)
    h.update(r.stdout.encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False) -> str:
    digest = source_hash()
    if not force and os.path.exists(LIB) and os.path.exists(HASH):
        with open(HASH) as f:
            if f.read().strip() == digest:
                return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fopenmp", "-o", tmp, *objs, "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(HASH + ".tmp", "w") as f:
        f.write(digest + "\n")
    os.replace(HASH + ".tmp", HASH)
    return LIB


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv, force="--force" in sys.argv))
