"""Builds libnepzbl.so (the C-ABI CUDA library) in-tree for sm_103a.

    python -m paper_2305_08140_gb300.build [--verbose]

The library is written to paper_2305_08140_gb300/lib/libnepzbl.so.  Only the
CUDA toolkit (nvcc) is needed; the build is a single nvcc invocation.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libnepzbl.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["nepzbl.cu", "nep_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "nepzbl.h"))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library unless it is newer than every source."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    tag = f"{os.getpid()}"
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
    if verbose:
        flags.append("-Xptxas=-v")
    # one object per translation unit, compiled in parallel, then linked
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(LIBDIR, src.replace(".cu", f".{tag}.o"))
        cmd = [_nvcc(), *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                            text=True)))
        objs.append(obj)
    errors = []
    for cmd, pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            errors.append(" ".join(cmd) + "\n" + out + err)
        elif verbose:
            sys.stderr.write(out + err)
    if errors:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + f".{tag}.tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="--verbose" in sys.argv)
    print(LIB)
