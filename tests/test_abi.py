"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/qcd.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(qcd_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["qcd_gauge_load", "qcd_clover_build", "qcd_dslash_eo", "qcd_clover_apply", "qcd_solve"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1709_08785_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_1709_08785_gb300 import qcd

    assert set(declared_functions()) <= set(qcd.EXPORTS) | {"qcd_solve_opts_default"}


def test_strerror_without_gpu():
    from paper_1709_08785_gb300 import build

    lib = ctypes.CDLL(build.build())
    lib.qcd_strerror.restype = ctypes.c_char_p
    assert lib.qcd_strerror(0) == b"ok"
    assert lib.qcd_strerror(-4) == b"not converged"
