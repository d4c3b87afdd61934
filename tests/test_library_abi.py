"""The C-ABI library builds, loads and exports every entry point include/omen.h declares.

No compute call is made (no GPU needed): only symbol presence and the binding's signatures.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(omen_[A-Za-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    from paper_1003_4570_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    return path


def test_header_declares_the_paper_calls():
    names = declared_entry_points()
    for required in ("omen_build_lattice", "omen_assemble_H", "omen_eigs", "omen_hx", "omen_create"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    import ctypes
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads(built_lib):
    from paper_1003_4570_gb300 import omen
    L = omen.lib()
    for n in declared_entry_points():
        assert hasattr(L, n)
