"""Builds libpmp.so, the CUDA library behind include/pmp.h, for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into ``paper_2509_18261_gb300/_lib/libpmp.so`` (CUDA runtime linked
statically).  Floating-point contraction is off on the device (-fmad=false)
and on the host (-ffp-contract=off): the library's arithmetic order is part of
its contract.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libpmp.so")
SOURCES = ["pmp_api.cu", "pmp_particles.cu", "pmp_mesh.cu", "pmp_sort.cu", "pmp_noalloc.cu", "pmp_batch.cu", "pmp_probe.cu", "pmp_exchange.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def cflags(verbose=False):
    f = ARCH + [
        "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
        "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
        "-I", os.path.join(ROOT, "include"), "-I", CSRC,
    ]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile (if stale) and return the path of libpmp.so."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "pmp.h"))
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc()] + cflags(verbose) + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    logs = []
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            logs = list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        # every symbol resolved at link time: a missing definition fails the build, not the first load
        run([nvcc()] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", LIB] + objs)
    if verbose:
        for line in logs:
            print(line)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
