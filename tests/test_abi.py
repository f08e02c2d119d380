"""The C ABI: the library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ddamg.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ddamg_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1303_1377_gb300 import build

    return build.build()


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for must in ("ddamg_setup", "ddamg_solve", "ddamg_apply_D", "ddamg_solve_batch", "ddamg_setup_from_vectors",
                 "ddamg_get_vectors", "ddamg_set_mass", "ddamg_set_stream", "ddamg_destroy", "ddamg_error_string"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_structs_match_header(libpath):
    from paper_1303_1377_gb300 import ddamg

    p = ddamg.default_params()
    # defaults are Table 1 of the paper
    assert (p.n_inv, p.n_vec, tuple(p.block), p.coarse_tol, p.n_kv, p.tol, p.nu, p.mr_steps, p.coarse_restart) == (
        6, 20, (4, 4, 4, 4), 5e-2, 25, 1e-10, 2, 4, 30)
    assert ddamg.lib.ddamg_error_string(-4) == b"not converged"
    # mixed-precision outer scheme (no counterpart in the paper)
    assert (p.outer, p.cycle_tol) == (ddamg.OUTER_REFINE, 1e-5)
    assert p.setup_update == ddamg.SETUP_DDALPHA  # Algorithm 2


def test_invalid_lattice_rejected_without_gpu_work(libpath):
    """Argument checks run before any CUDA call: odd block counts are refused."""
    import numpy as np

    from paper_1303_1377_gb300 import ddamg

    p = ddamg.default_params(block=(4, 4, 4, 4))
    U = np.zeros((12 ** 4, 4, 3, 3), dtype=np.complex128)
    with pytest.raises(ddamg.DDAMGError) as e:
        ddamg.Solver((12, 12, 12, 12), U, 0.0, 1.0, p, setup=False)
    assert e.value.status == -1


@pytest.mark.parametrize("kw", [{"outer": 2}, {"cycle_tol": 0.0}, {"cycle_tol": 1.0}, {"setup_update": 2}])
def test_invalid_outer_scheme_rejected_without_gpu_work(libpath, kw):
    import numpy as np

    from paper_1303_1377_gb300 import ddamg

    p = ddamg.default_params(block=(2, 2, 2, 2), **kw)
    U = np.zeros((4 ** 4, 4, 3, 3), dtype=np.complex128)
    with pytest.raises(ddamg.DDAMGError) as e:
        ddamg.Solver((4, 4, 4, 4), U, 0.0, 1.0, p, setup=False)
    assert e.value.status == -1 and "cycle_tol" in str(e.value)


def test_struct_layouts_match_the_compiled_header(tmp_path):
    """Size and every field offset of the ABI structs, as a C compiler lays them out from
    include/ddamg.h, equal those of the ctypes binding."""
    import shutil
    import subprocess

    from paper_1303_1377_gb300 import ddamg

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ddamg_lattice": ddamg.Lattice, "ddamg_params": ddamg.Params, "ddamg_stats": ddamg.Stats,
               "ddamg_kernel_profile": ddamg.KernelProfile, "ddamg_ml_params": ddamg.MLParams}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ddamg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_third_level_defaults_and_argument_checks(libpath):
    """ddamg_ml_default_params, and the third-level calls refuse a null handle before any CUDA work."""
    from paper_1303_1377_gb300 import ddamg

    p = ddamg.ml_default_params()
    assert (tuple(p.block1), p.n_vec1, p.nu1, p.mr_steps1, p.inner, p.inner_kv, p.inner_tol, p.coarse_tol, p.coarse_restart) == (
        (2, 2, 2, 2), 20, 2, 4, 0, 10, 5e-2, 5e-2, 30)
    assert (p.n_inv1, p.setup_update1) == (6, ddamg.SETUP_DDALPHA)
    assert ddamg.lib.ddamg_ml_build(None, ctypes.byref(p), None) == -1
    assert ddamg.lib.ddamg_ml_solve(None, None, None, 1, 1e-10, None) == -1
    assert ddamg.lib.ddamg_ml_release(None) == -1
    assert ddamg.lib.ddamg_ml_setup(None, ctypes.byref(p), None, None) == -1
    assert ddamg.lib.ddamg_ml_add_level(None, ctypes.byref(p), None, 1, None) == -1
    assert ddamg.lib.ddamg_ml_levels(None) == -1
