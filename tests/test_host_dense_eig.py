"""The library's host dense linear algebra (projected Lanczos problems) on the CPU.

`csrc/dense_eig.cpp` is plain C++: it is compiled here with the host compiler behind a small
C shim and checked against LAPACK (numpy) — eigenvalues, backward error and orthogonality of
the eigenvectors on random, degenerate, graded, already-diagonal and nearly-split tridiagonal
matrices; the Cholesky factor and the triangular inverse by their defining identities.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1003_4570_gb300", "csrc")

SHIM = r"""
#include <complex>
#include "dense_eig.h"
using cd = std::complex<double>;
extern "C" int t_heig(int n, const double* A, double* w, double* Z) {
  return hermitian_eig(n, reinterpret_cast<const cd*>(A), w, reinterpret_cast<cd*>(Z));
}
extern "C" int t_chol(int b, const double* G, double* R) {
  return cholesky_upper(b, reinterpret_cast<const cd*>(G), reinterpret_cast<cd*>(R));
}
extern "C" void t_uinv(int b, const double* R, double* Ri) {
  upper_inverse(b, reinterpret_cast<const cd*>(R), reinterpret_cast<cd*>(Ri));
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("dense")
    (d / "shim.cpp").write_text(SHIM)
    so = d / "libdense.so"
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, os.path.join(CSRC, "dense_eig.cpp"),
                    str(d / "shim.cpp"), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    p = ctypes.c_void_p
    L.t_heig.argtypes = [ctypes.c_int, p, p, p]
    L.t_chol.argtypes = [ctypes.c_int, p, p]
    L.t_uinv.argtypes = [ctypes.c_int, p, p]
    L.t_uinv.restype = None
    return L


def heig(L, A):
    n = A.shape[0]
    Af = np.asfortranarray(A.astype(np.complex128))
    w = np.zeros(n)
    Z = np.zeros((n, n), dtype=np.complex128, order="F")
    assert L.t_heig(n, Af.ctypes.data, w.ctypes.data, Z.ctypes.data) == 0
    return w, Z


def check_eig(L, A, rtol=1e-13):
    n = A.shape[0]
    w, Z = heig(L, A)
    ref = np.linalg.eigvalsh(A)
    scale = max(np.abs(ref).max(), 1e-300)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(w - ref).max() <= rtol * n * scale
    assert np.abs(A @ Z - Z * w[None, :]).max() <= rtol * n * scale
    assert np.abs(Z.conj().T @ Z - np.eye(n)).max() <= rtol * n


def rand_herm(n, seed, cplx=True):
    g = np.random.default_rng(seed)
    B = g.standard_normal((n, n)) + (1j * g.standard_normal((n, n)) if cplx else 0)
    return (B + B.conj().T) / 2


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 200])
def test_random_hermitian(lib, n):
    check_eig(lib, rand_herm(n, n))
    check_eig(lib, rand_herm(n, n + 1, cplx=False).astype(np.complex128))


def test_degenerate_and_structured(lib):
    g = np.random.default_rng(3)
    Q, _ = np.linalg.qr(g.standard_normal((40, 40)) + 1j * g.standard_normal((40, 40)))
    lam = np.repeat([-2.0, 0.5, 0.5 + 1e-13, 3.0], 10)
    check_eig(lib, (Q * lam[None, :]) @ Q.conj().T)
    check_eig(lib, np.diag(np.linspace(-1, 1, 30)).astype(complex))          # already diagonal
    check_eig(lib, np.eye(25, dtype=complex))                               # one 25-fold value
    # graded: entries from 1e-8 to 1e4
    D = np.diag(np.logspace(-4, 2, 20))
    check_eig(lib, D @ rand_herm(20, 5) @ D)


def test_nearly_split_tridiagonal(lib):
    """Lanczos matrices: a converged Ritz value shows up as a tiny off-diagonal entry."""
    g = np.random.default_rng(7)
    n = 120
    a = g.standard_normal(n)
    b = np.abs(g.standard_normal(n - 1))
    b[[10, 50, 51, 90]] = [1e-15, 1e-12, 0.0, 1e-17]
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    check_eig(lib, T.astype(complex))


def test_cholesky_and_triangular_inverse(lib):
    for b, seed in ((1, 1), (4, 2), (16, 3)):
        g = np.random.default_rng(seed)
        B = g.standard_normal((3 * b, b)) + 1j * g.standard_normal((3 * b, b))
        G = np.asfortranarray(B.conj().T @ B)
        R = np.zeros((b, b), dtype=np.complex128, order="F")
        assert lib.t_chol(b, G.ctypes.data, R.ctypes.data) == 0
        assert np.allclose(np.tril(R, -1), 0)
        assert np.all(np.real(np.diag(R)) > 0)
        assert np.abs(R.conj().T @ R - G).max() <= 1e-13 * np.abs(G).max()
        Ri = np.zeros((b, b), dtype=np.complex128, order="F")
        lib.t_uinv(b, R.ctypes.data, Ri.ctypes.data)
        assert np.abs(R @ Ri - np.eye(b)).max() <= 1e-12 * np.linalg.cond(R)
    # not positive definite: reported, not factored
    G = np.asfortranarray(np.diag([1.0, -1.0, 2.0]).astype(complex))
    R = np.zeros((3, 3), dtype=np.complex128, order="F")
    assert lib.t_chol(3, G.ctypes.data, R.ctypes.data) != 0
