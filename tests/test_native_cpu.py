"""The native library without a GPU: it builds for sm_103a, loads, exports
every entry point that include/fempic.h declares, its ctypes structures match
the C layouts, and host-side validation returns error codes (no compute)."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fempic.h")


@pytest.fixture(scope="module")
def native():
    from paper_2111_12411_gb300 import build
    build.build()
    from paper_2111_12411_gb300 import native as nat
    nat.load()
    return nat


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(femPIC_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol(native):
    lib = native.load()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(n for n, _, _ in native.EXPORTS) == names


def test_struct_layouts_match_c(native, tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text('#include "fempic.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(femPIC_mesh),'
                    ' sizeof(femPIC_species), sizeof(femPIC_opts), sizeof(femPIC_diag),'
                    ' sizeof(femPIC_info), offsetof(femPIC_opts, stream), offsetof(femPIC_info, device_bytes),'
                    ' offsetof(femPIC_info, device_allocations), offsetof(femPIC_info, cg_smooth_degree));'
                    'return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(native.femPIC_mesh), ctypes.sizeof(native.femPIC_species),
            ctypes.sizeof(native.femPIC_opts), ctypes.sizeof(native.femPIC_diag),
            ctypes.sizeof(native.femPIC_info), native.femPIC_opts.stream.offset,
            native.femPIC_info.device_bytes.offset, native.femPIC_info.device_allocations.offset,
            native.femPIC_info.cg_smooth_degree.offset]
    assert got == want


def test_extension_struct_layouts_match_c(native, tmp_path):
    prog = tmp_path / "sizes2.c"
    prog.write_text('#include "fempic.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(femPIC_projection),'
                    ' sizeof(femPIC_injector), sizeof(femPIC_batch_tuning), offsetof(femPIC_injector, v_sigma),'
                    ' offsetof(femPIC_batch_tuning, particle_ms), offsetof(femPIC_diag, divb_ref));return 0;}\n')
    exe = tmp_path / "sizes2"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(native.femPIC_projection), ctypes.sizeof(native.femPIC_injector),
            ctypes.sizeof(native.femPIC_batch_tuning), native.femPIC_injector.v_sigma.offset,
            native.femPIC_batch_tuning.particle_ms.offset, native.femPIC_diag.divb_ref.offset]
    assert got == want


def test_constants_match_header(native):
    src = open(HEADER).read()
    m = re.search(r"#define\s+FEMPIC_PROBE_MAX_POINTS\s+(\d+)", src)
    assert m and int(m.group(1)) == native.FEMPIC_PROBE_MAX_POINTS
    codes = dict(re.findall(r"#define\s+(FEMPIC_ERR_\w+)\s+\(?(-?\d+)\)?", src))
    codes.update(re.findall(r"(FEMPIC_ERR_\w+)\s*=\s*(-?\d+)", src))
    for name, val in codes.items():
        if hasattr(native, name):
            assert getattr(native, name) == int(val), name


def test_default_opts(native):
    o = native.default_opts()
    assert o.precision == 1 and o.scheme == 0 and o.cg_rtol == 1e-12 and o.sort_period == 1
    assert abs(o.beta - 0.25) < 1e-15 and abs(o.gamma - 0.5) < 1e-15


def _small():
    xyz, tets = workloads.kuhn_box(2, 2, 2, jitter=0.1, seed=3)
    rng = np.random.default_rng(0)
    x, tet = workloads.sample_uniform_in_tets(xyz, tets, 10, rng)
    return xyz, tets, x, tet


def test_host_validation_errors(native):
    xyz, tets, x, tet = _small()
    v = np.zeros_like(x)
    bad = tets.copy()
    bad[3, 1] = bad[3, 0]  # repeated vertex
    with pytest.raises(native.FemPICError) as ei:
        native.femPIC_create(xyz, bad, 1, -1.6e-19, 9.1e-31, 1.0, x, v, tet)
    assert ei.value.code == native.FEMPIC_ERR_MESH
    flat = xyz.copy()
    flat[:, 2] = 0.0  # every tet degenerate
    with pytest.raises(native.FemPICError) as ei:
        native.femPIC_create(flat, tets, 1, -1.6e-19, 9.1e-31, 1.0, x, v, tet)
    assert ei.value.code == native.FEMPIC_ERR_MESH
    with pytest.raises(native.FemPICError) as ei:
        native.femPIC_create(xyz, tets, 4, -1.6e-19, 9.1e-31, 1.0, x, v, tet)
    assert ei.value.code == native.FEMPIC_ERR_ARG
    o = native.default_opts()
    o.push = native.PUSH["ab4"]
    with pytest.raises(native.FemPICError) as ei:  # the Adams-Bashforth push stops at order 2
        native.femPIC_create(xyz, tets, 3, -1.6e-19, 9.1e-31, 1.0, x, v, tet, o)
    assert ei.value.code == native.FEMPIC_ERR_ARG
    wrong = (tet + 1) % len(tets)
    with pytest.raises(native.FemPICError) as ei:
        native.femPIC_create(xyz, tets, 1, -1.6e-19, 9.1e-31, 1.0, x, v, wrong)
    assert ei.value.code == native.FEMPIC_ERR_ARG
    species = [dict(q=-1.6e-19, m=9.1e-31, weight=1.0, x=x, v=v, tet=tet)]
    with pytest.raises(native.FemPICError) as ei:  # face tags are 0..7
        native.femPIC_create_ext(xyz, tets, 1, species, np.full((len(tets), 4), 8, dtype=np.int32))
    assert ei.value.code == native.FEMPIC_ERR_ARG
    with pytest.raises(native.FemPICError) as ei:  # absorbing walls and the Adams-Bashforth push
        native.femPIC_create_ext(xyz, tets, 1, species, np.full((len(tets), 4), 2, dtype=np.int32), o)
    assert ei.value.code == native.FEMPIC_ERR_ARG
    vnan = v.copy()
    vnan[4, 1] = np.nan  # a non-finite velocity is refused on the host
    with pytest.raises(native.FemPICError) as ei:
        native.femPIC_create(xyz, tets, 1, -1.6e-19, 9.1e-31, 1.0, x, vnan, tet)
    assert ei.value.code == native.FEMPIC_ERR_ARG and "velocity" in str(ei.value)
    xinf = x.copy()
    xinf[2, 0] = np.inf  # and a position that is not inside its tet
    with pytest.raises(native.FemPICError) as ei:
        native.femPIC_create(xyz, tets, 1, -1.6e-19, 9.1e-31, 1.0, xinf, v, tet)
    assert ei.value.code == native.FEMPIC_ERR_ARG
    nonman = np.vstack([tets, tets[:1]])  # a face shared by three tets
    with pytest.raises(native.FemPICError) as ei:
        native.femPIC_create(xyz, nonman, 1, -1.6e-19, 9.1e-31, 1.0, x, v, tet)
    assert ei.value.code == native.FEMPIC_ERR_MESH


def test_product_never_reaches_the_oracle():
    """The library package imports nothing from the oracle (only the tests,
    smoke() and the benchmark's CPU-baseline and reference arms may), and its
    binding refuses to run without the built library instead of falling back."""
    import ast
    pkg = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2111_12411_gb300")
    for name in os.listdir(pkg):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, name)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert not any(a.name.split(".")[0] == "oracle" for a in node.names), name
            elif isinstance(node, ast.ImportFrom):
                assert (node.module or "").split(".")[0] != "oracle", name
    from paper_2111_12411_gb300 import native as nat
    saved, nat._lib = nat._lib, None
    try:
        with pytest.raises(ImportError):
            nat.load(os.path.join(pkg, "no_such_library.so"))
    finally:
        nat._lib = saved
