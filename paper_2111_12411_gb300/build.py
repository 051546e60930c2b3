"""Build the native library ``libfempic.so`` in-tree for sm_103a.

Two translation units, compiled in parallel:
* ``csrc/setup.cpp`` (host set-up; no floating-point contraction, so the
  barycentric maps are rounded exactly as written),
* ``csrc/fempic.cu`` (kernels and the C ABI), ``nvcc -gencode
  arch=compute_103a,code=sm_103a -lineinfo``.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfempic.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(INCLUDE, "fempic.h")]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    return p.stdout + p.stderr


def build(force=False, verbose=False, ptxas_info=False):
    """Compile the library if any source is newer than it; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    host_o = os.path.join(BUILD, "setup.o")
    dev_o = os.path.join(BUILD, "fempic.o")
    cmds = [
        ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I" + INCLUDE, "-c",
         os.path.join(CSRC, "setup.cpp"), "-o", host_o],
        [nvcc, "-O3", "-std=c++17", "-lineinfo", ARCH, "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I" + INCLUDE, "-c", os.path.join(CSRC, "fempic.cu"), "-o", dev_o]
        + os.environ.get("FEMPIC_NVCC_FLAGS", "").split()
        + (["-Xptxas", "-v"] if ptxas_info else []),
    ]
    with ThreadPoolExecutor(2) as ex:
        outs = list(ex.map(lambda c: _run(c, verbose), cmds))
    if ptxas_info:
        print(outs[1])
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", ARCH, "-o", tmp, host_o, dev_o, "-lpthread"], verbose)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
