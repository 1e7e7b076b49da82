"""Builds ``libmetricgraph.so`` in-tree with nvcc for sm_103a.

Four translation units compiled in parallel and linked into one shared
library next to this file:

* ``em_step_f32.cu``  binary32-mixed kernels (FMA contraction allowed)
* ``em_step_f64.cu``  binary64 kernels, ``--fmad=false`` so every operation
                      rounds as written
* ``mg_api.cpp``      the C ABI (host), ``-ffp-contract=off`` so the jump
                      thresholds round identically on x86-64 and AArch64
* ``mg_noalloc.cu``   the histogram entry point that allocates nothing
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmetricgraph.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

UNITS = [
    ("em_step_f32.cu", []),
    ("em_step_f64.cu", ["--fmad=false"]),
    ("mg_api.cpp", ["-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-pthread"]),
    ("mg_noalloc.cu", []),
]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmetricgraph")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link the library; returns its path.  Raises on failure."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    procs, objs = [], []
    for src, extra in UNITS:
        # per-process object names: concurrent builds (test workers) do not
        # overwrite each other's objects; the library is replaced atomically
        obj = os.path.join(BUILD, f"{src.rsplit('.', 1)[0]}.{os.getpid()}.o")
        cmd = [nvcc, *ARCH, *common, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info and src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    logs = []
    for src, pr in procs:
        out, _ = pr.communicate()
        logs.append(out.decode(errors="replace"))
        if pr.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{out.decode(errors='replace')}")
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout.decode(errors='replace')}")
    os.replace(tmp, LIB)
    for obj in objs:
        try:
            os.remove(obj)
        except OSError:
            pass
    if verbose or ptxas_info:
        print("\n".join(logs), file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
