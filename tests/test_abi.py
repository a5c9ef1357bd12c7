"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/fsmlmc.h declares (no GPU needed: nothing is called)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fsmlmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
    src = re.sub(r"\{[^{}]*\}", ";", src)  # drop struct / enum bodies
    names = set()
    for stmt in src.split(";"):
        stmt = " ".join(stmt.split())
        if "(" not in stmt or stmt.startswith(("typedef", "enum", "struct", "extern")):
            continue
        m = re.match(r"^[A-Za-z_][A-Za-z0-9_ ]*?[\s*]+([A-Za-z_][A-Za-z0-9_]*)\s*\(", stmt)
        if m:
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2212_04430_gb300 import fsmlmc
    return ctypes.CDLL(fsmlmc.LIB_PATH)


def test_header_declares_the_paper_operations():
    names = declared_functions()
    for n in ("wilson_dslash", "shifted_solve", "mlmc_level_trace", "variance_sample"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2212_04430_gb300 import fsmlmc
    assert set(declared_functions()) == set(fsmlmc.EXPORTS)


def test_library_is_sm103a_only(lib):
    """The fat binary holds sm_103a code only (no PTX for JIT on other parts)."""
    from paper_2212_04430_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
