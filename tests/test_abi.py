"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(nbm_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("nbm_init_problem", "nbm_destroy", "nbm_residual", "nbm_loss_grad",
              "nbm_train_steps", "nbm_eval_grid", "nbm_grid_cg_solve", "nbm_last_error"):
        assert n in names


def test_library_loads_and_exports_all_symbols():
    from paper_2210_14907_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_invalid_descriptor_is_rejected_without_a_gpu():
    import paper_2210_14907_gb300 as nbm
    lib = nbm.load_library()
    d = nbm.ProblemDesc(width=96).to_c()
    h = ctypes.c_void_p()
    rc = lib.nbm_init_problem(ctypes.byref(d), ctypes.byref(h))
    assert rc == 1 and h.value is None
    assert b"width" in lib.nbm_last_error()


@pytest.mark.parametrize("field,value,word", [("grid_jump", 3, b"grid_jump"),
                                              ("grid_jump", -1, b"grid_jump"),
                                              ("reserved0", 1, b"reserved0"),
                                              ("refine_levels", 4, b"refine_levels"),
                                              ("activation", 2, b"activation")])
def test_descriptor_fields_are_validated_without_a_gpu(field, value, word):
    import paper_2210_14907_gb300 as nbm
    lib = nbm.load_library()
    d = nbm.ProblemDesc().to_c()
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.nbm_init_problem(ctypes.byref(d), ctypes.byref(h)) == 1 and h.value is None
    assert word in lib.nbm_last_error()


def test_descriptor_layout_matches_the_header():
    """The ctypes mirror has the C struct's size: every field in order, no
    padding surprises (int32 tail padded to 8 bytes)."""
    import paper_2210_14907_gb300 as nbm
    assert ctypes.sizeof(nbm._Desc) == 4 * 4 + 11 * 8 + 6 * 4


def test_grid_entry_points_reject_null_arguments_without_a_gpu():
    import paper_2210_14907_gb300 as nbm
    lib = nbm.load_library()
    for fn in (lib.nbm_grid_cg_solve, lib.nbm_grid_solve_refined):
        assert fn(None, 16, 1e-10, 100, None, None, None, None) == 1
        assert b"NULL" in lib.nbm_last_error()
    ps, dj, fb = ctypes.c_int(-1), ctypes.c_double(-1.0), ctypes.c_int(-1)
    assert lib.nbm_grid_last_jump_info(ctypes.byref(ps), ctypes.byref(dj), ctypes.byref(fb)) == 0
    assert ps.value >= 0 and fb.value in (0, 1)
    assert lib.nbm_grid_last_jump_info(None, None, None) == 0


def test_header_compiles_as_c_and_agrees_with_the_binding(tmp_path):
    """include/nbm.h is plain C: a C11 program includes it, links libnbm.so and
    calls it.  Every field offset of nbm_problem_desc matches the ctypes mirror
    of the Python binding, and an invalid descriptor is refused from C (status
    NBM_ERR_INVALID_ARG, *out set to NULL) without a GPU."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import paper_2210_14907_gb300 as nbm
    from paper_2210_14907_gb300 import build
    libdir = os.path.dirname(build.build())
    names = [f[0] for f in nbm._Desc._fields_]
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "nbm.h"', "int main(void) {",
           '  printf("size %zu\\n", sizeof(nbm_problem_desc));']
    src += [f'  printf("{n} %zu\\n", offsetof(nbm_problem_desc, {n}));' for n in names]
    src += ["  nbm_problem_desc d = {0};", "  d.geometry = NBM_GEOM_SPHERE;", "  d.n_hidden = 2;",
            "  d.width = 96;",
            "  nbm_problem* p = (nbm_problem*)&d;",
            "  int rc = nbm_init_problem(&d, &p);",
            '  printf("rc %d %d\\n", rc, p == NULL);',
            '  printf("count %lld\\n", (long long)nbm_param_count(NULL));',
            '  printf("msg %s\\n", nbm_last_error());',
            "  return 0;", "}"]
    c = tmp_path / "abi.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(c), "-o", str(exe), "-L", libdir, "-lnbm",
                    "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    vals = dict(line.split(" ", 1) for line in out.splitlines() if line)
    assert int(vals["size"]) == ctypes.sizeof(nbm._Desc)
    for n in names:
        assert int(vals[n]) == getattr(nbm._Desc, n).offset, n
    assert vals["rc"] == "1 1"
    assert vals["count"] == "-1"
    assert "width" in vals["msg"]
