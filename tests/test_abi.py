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
