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


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    return p.stdout + p.stderr


# Test variants of the library, built beside the default one:
# * "checked": every index taken from a caller or a table is range-checked
#   (FEMPIC_ERR_BOUNDS instead of an out-of-range access);
# * "barrier_test": the grid barrier's spin limit lowered to 2e5 polls and one
#   CTA of every persistent CG launch made absent from its barriers, so the
#   others' bounded waits run out and the launch returns FEMPIC_ERR_BARRIER.
VARIANTS = {
    "checked": ["-DFEMPIC_CHECKS=1"],
    "barrier_test": ["-DFEMPIC_BARRIER_SPIN_LIMIT=200000", "-DFEMPIC_TEST_ABSENT_CTA=1"],
}


def variant_path(variant):
    return LIB if variant is None else os.path.join(HERE, f"libfempic_{variant}.so")


def build(force=False, verbose=False, ptxas_info=False, variant=None):
    """Compile the library (or one of its test variants) if any source is newer
    than it; returns its path."""
    lib_path = variant_path(variant)
    if not force and not _stale(lib_path):
        return lib_path
    bdir = BUILD if variant is None else os.path.join(BUILD, variant)
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    host_o = os.path.join(bdir, "setup.o")
    dev_o = os.path.join(bdir, "fempic.o")
    cmds = [
        ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I" + INCLUDE, "-c",
         os.path.join(CSRC, "setup.cpp"), "-o", host_o],
        [nvcc, "-O3", "-std=c++17", "-lineinfo", ARCH, "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I" + INCLUDE, "-c", os.path.join(CSRC, "fempic.cu"), "-o", dev_o]
        + (VARIANTS[variant] if variant else os.environ.get("FEMPIC_NVCC_FLAGS", "").split())
        + (["-Xptxas", "-v"] if ptxas_info else []),
    ]
    with ThreadPoolExecutor(2) as ex:
        outs = list(ex.map(lambda c: _run(c, verbose), cmds))
    if ptxas_info:
        print(outs[1])
    tmp = lib_path + ".tmp"
    _run([nvcc, "-shared", ARCH, "-o", tmp, host_o, dev_o, "-lpthread"], verbose)
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
