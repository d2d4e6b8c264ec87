"""Build the CUDA library in place: paper_1903_03406_gb300/libcdr.so (sm_103a).

The translation units (the kernels, the host driver and the no-allocation
predicate entry point) compile in parallel with nvcc; host code is compiled without floating-point contraction so that the
host-side FP64 set-up (facet reference points, the shortest-edge guard) rounds
exactly as written.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcdr.so")
SOURCES = ["kernels.cu", "api.cu", "noalloc.cu"]
HEADERS = ["kernels.cuh", "mesh.cuh", "predicates.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _flags():
    f = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-diag-suppress", "1444"]
    if os.environ.get("CDR_CHECKED"):
        f.append("-DCDR_CHECKED")  # bounds-checked diagnostic build
    if os.environ.get("CDR_PHASES"):
        f.append("-DCDR_PHASES")  # per-phase timing of region growth (diagnostic build)
    # build-time sizes of the growth workspaces (CDR_T1_CAPB, CDR_T1_HCAP,
    # CDR_G1_MINB), e.g. CDR_DEFS="CDR_T1_HCAP=512 CDR_G1_MINB=4"
    f += ["-D" + d for d in os.environ.get("CDR_DEFS", "").split()]
    return f


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "cdr.h"))
    return all(os.path.getmtime(d) <= t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc()] + _flags() + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc(), ARCH, "-shared", "-o", tmp] + objs
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
