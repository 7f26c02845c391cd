"""The C-ABI library builds, loads and exports every entry point include/bltc.h declares.

No compute call is made here (no GPU is needed); the GPU tests call through the same ABI.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bltc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:[\w\*]+\s+)+\**(bltc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2003_01836_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("bltc_context_create", "bltc_tree_build", "bltc_lists_build",
                 "bltc_modified_charges", "bltc_evaluate", "bltc_solve", "bltc_solve_host",
                 "bltc_direct_sum", "bltc_tree_export", "bltc_lists_export", "bltc_stats"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_functions():
        assert hasattr(built_lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_2003_01836_gb300 as b
    assert set(declared_functions()) <= set(b.exported_symbols())
    for name in declared_functions():
        assert callable(getattr(b, name)), name


def test_version_without_gpu(built_lib):
    built_lib.bltc_version.restype = ctypes.c_int
    assert built_lib.bltc_version() == 1


def test_params_layout_matches_header():
    import paper_2003_01836_gb300 as b
    assert ctypes.sizeof(b.bltc_params) == 40
    assert b.bltc_params.theta.offset == 24 and b.bltc_params.kappa.offset == 32
