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


STRUCTS = {
    "LatticeDesc": "omen_lattice_desc", "TBParams": "omen_tb_params", "HamOpts": "omen_ham_opts",
    "EigOpts": "omen_eig_opts", "EigInfo": "omen_eig_info", "Grid": "omen_grid", "CGOpts": "omen_cg_opts",
    "TuneResult": "omen_tune_result", "SolveInfo": "omen_solve_info", "SCFDesc": "omen_scf_desc",
    "SCFInfo": "omen_scf_info", "EffMassDesc": "omen_effmass_desc", "MLPDesc": "omen_mlp_desc",
    "KbatchItem": "omen_kbatch_item", "VFFParams": "omen_vff_params", "VFFOpts": "omen_vff_opts",
    "VFFInfo": "omen_vff_info", "FrozenStates": "omen_frozen_states", "NewtonOpts": "omen_newton_opts",
    "NewtonInfo": "omen_newton_info",
}


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets the C compiler gives
    the header's struct of the same name (a field renamed, reordered or retyped on one side
    fails here instead of corrupting arguments at run time)."""
    import ctypes
    import shutil
    import subprocess
    from paper_1003_4570_gb300 import omen
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "omen.h"', "int main(void) {"]
    expected = []
    for py, c in STRUCTS.items():
        cls = getattr(omen, py)
        lines.append(f'  printf("%zu\\n", sizeof({c}));')
        expected.append(ctypes.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({c}, {name}));')
            expected.append(getattr(cls, name).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expected


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the shared library missing, the first call raises."""
    from paper_1003_4570_gb300 import omen
    monkeypatch.setattr(omen, "_lib", None)
    monkeypatch.setattr(omen, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        omen.lib()


def test_binding_refuses_buffers_smaller_than_the_call_uses():
    """Too small a buffer is refused in the binding, before the library could read or write past
    its end; raw addresses pass unchecked."""
    import numpy as np
    from paper_1003_4570_gb300 import omen
    ham = object.__new__(omen.Hamiltonian)
    ham.handle = None
    ham.nrows, ham.is_complex, ham.elem_bytes, ham.precision = 1000, True, 8, omen.OMEN_F32_REFINE64
    assert ham.evec_bytes == 16                      # refined solves return complex128
    ham.precision = omen.OMEN_F32
    assert ham.evec_bytes == 8
    small = np.zeros(2 * 1000 - 1, dtype=np.complex64)
    with pytest.raises(ValueError):
        omen.omen_hx(None, ham, small, small, nvec=2)
    with pytest.raises(ValueError):
        omen.omen_eigs(None, ham, 4, evecs_dev=np.zeros((3, 1000), dtype=np.complex64))
    with pytest.raises(ValueError):
        omen.omen_density_accum(None, ham, np.zeros((2, 1000), dtype=np.complex64), 2, [1.0, 1.0], 1.0, None)
    with pytest.raises(ValueError):
        omen.omen_hx_kbatch(None, ham, np.zeros((3, 3)), np.zeros(2999, np.complex64), np.zeros(3000, np.complex64))
    assert omen._nbytes(12345) is None and omen._nbytes(np.zeros(4)) == 32
