"""Host-core CSR product of the oracle's matrices (oracle; test infrastructure).

`matvec(A, x, threads)` runs the plain C loop in csr_matvec.c over A's rows (OpenMP, one row
per iteration, each row summed in index order).  It computes exactly what `A @ x` computes;
it exists so that the oracle's repeated product (H·X inside Lanczos, Section II-B) can be
timed on all host cores.  The shared object is compiled from csr_matvec.c with the system C
compiler on first use (or by the package build step) next to this file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csr_matvec.c")
_LIB = os.path.join(_HERE, "libcsr_matvec.so")
_lib = None


def build(force=False) -> str:
    """Compile csr_matvec.c (gcc -O2 -fopenmp, no FMA contraction, so a row's products and sums
    round as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.oracle_csr_matvec.restype = None
        L.oracle_csr_matvec.argtypes = [C.c_longlong] + [C.c_void_p] * 5 + [C.c_int]
        L.oracle_max_threads.restype = C.c_int
        _lib = L
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def matvec(A, x, threads: int = 0, out=None):
    """y = A x for a real scipy CSR matrix with 32-bit indices."""
    L = _load()
    A = A.tocsr()
    if A.indptr.dtype != np.int32 or A.indices.dtype != np.int32:
        raise ValueError("32-bit CSR indices expected")
    data = np.ascontiguousarray(A.data, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.shape[0]) if out is None else out
    L.oracle_csr_matvec(A.shape[0], A.indptr.ctypes.data, A.indices.ctypes.data, data.ctypes.data, x.ctypes.data,
                        y.ctypes.data, int(threads))
    return y
