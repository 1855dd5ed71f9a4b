"""The C-ABI library builds, loads and exports every entry point that
include/abd.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

from paper_2201_10022_gb300 import abd, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(abd_[a-z_0-9]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert {"abd_create_scene", "abd_energy_grad_hess", "abd_solve", "abd_ccd_toi", "abd_step",
            "abd_destroy"} <= names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(abd.EXPORTS) <= names


def test_binding_signatures_load():
    L = abd.load()
    for n in abd.EXPORTS:
        assert getattr(L, n).argtypes is not None or n == "abd_last_error"


def test_default_params_through_the_struct_layout():
    """abd_default_params is host-only: reading its fields back through the
    binding's ctypes mirror checks the struct layout field by field"""
    p = abd.abd_default_params()
    assert p.dt == 0.01 and p.dhat == 1e-3 and p.kappa == 1e8
    assert list(p.gravity) == [0.0, 0.0, -9.8]
    assert p.mu == 0.0 and p.eps_v == 1e-3 and p.newton_tol == 0.0 and p.pcg_rel_tol == 1e-4
    assert p.ls_slack_rel == 1e-12 and p.ccd_s == 0.1
    assert (p.newton_max, p.pcg_max, p.ls_max, p.ccd_max) == (500, 20000, 30, 10000)
    assert p.precision == 0 and p.dense_max_dofs == 0


def test_host_side_argument_checks():
    L = abd.load()
    t = abd.abd_tuning()
    assert L.abd_get_tuning(None, ctypes.byref(t)) == 1  # ABD_ERR_INVALID_ARG
    t.grid_div = 0
    assert L.abd_set_tuning(None, ctypes.byref(t)) == 1
