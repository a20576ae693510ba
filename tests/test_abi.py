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
