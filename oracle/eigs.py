"""Eigenpairs of the tight-binding Hamiltonian (oracle; test infrastructure).

The paper (Section III-A item 1) solves the Schrödinger equation with an iterative
eigensolver, "(block) Lanczos or PARPACK"; its benchmark unit is 500 Lanczos iterations
(Section II-B).  The defined result is the set of eigenpairs of H; the oracle computes it by
a dense Hermitian eigensolve where that fits, and otherwise by plain Lanczos with full
reorthogonalisation (Lanczos 1950; Golub & Van Loan, Matrix Computations, Sec. 10.1),
applied to H for the lowest eigenvalues or to (H - sigma)^2 for those nearest sigma
(folded spectrum, Wang & Zunger 1994), with the eigenvalues of H taken as Rayleigh quotients.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def dense_eigh(H, subset=None):
    """All (or subset_by_index) eigenpairs of a Hermitian matrix, ascending."""
    A = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    return sla.eigh(A, subset_by_index=subset)


def nearest(evals, sigma, nev):
    """The nev eigenvalues closest to sigma (ties broken by value), sorted ascending."""
    evals = np.asarray(evals)
    order = np.lexsort((evals, np.abs(evals - sigma)))
    return np.sort(evals[order[:nev]])


def lanczos(apply, n, nev, v0, maxiter=2000, tol=1e-10, dtype=float):
    """Plain Lanczos with full (twice-applied Gram–Schmidt) reorthogonalisation.

    Returns the nev smallest Ritz values and vectors of the operator `apply` once the bound
    beta_m |s_{m,i}| on each of their residuals is below tol, or after maxiter steps.
    """
    V = np.zeros((maxiter + 1, n), dtype=dtype)
    alpha = np.zeros(maxiter)
    beta = np.zeros(maxiter)
    v = np.asarray(v0, dtype=dtype)
    V[0] = v / np.linalg.norm(v)
    m = 0
    theta = S = None
    for j in range(maxiter):
        w = apply(V[j])
        alpha[j] = np.real(np.vdot(V[j], w))
        for _ in range(2):                     # full reorthogonalisation, twice
            w = w - V[:j + 1].T @ (V[:j + 1].conj() @ w)
        beta[j] = np.linalg.norm(w)
        m = j + 1
        if m >= nev and (m % 10 == 0 or beta[j] < 1e-14 or m == maxiter):
            theta, S = sla.eigh_tridiagonal(alpha[:m], beta[:m - 1])
            resid = beta[j] * np.abs(S[-1, :nev])
            if np.all(resid < tol) or beta[j] < 1e-14:
                break
        if beta[j] < 1e-14:
            break
        V[j + 1] = w / beta[j]
    if theta is None or len(theta) != m:
        theta, S = sla.eigh_tridiagonal(alpha[:m], beta[:m - 1])
    X = V[:m].T @ S[:, :nev]
    return theta[:nev], X, m


def lowest(H, nev, v0, **kw):
    """Lowest nev eigenpairs of sparse H by plain Lanczos."""
    return lanczos(lambda x: H @ x, H.shape[0], nev, v0, dtype=H.dtype, **kw)


def folded(H, sigma, nev, v0, **kw):
    """nev eigenpairs of H nearest sigma by Lanczos on (H - sigma)^2.

    Eigenvalues are the Rayleigh quotients <x, H x> of the converged Ritz vectors.
    """
    def apply(x):
        y = H @ x - sigma * x
        return H @ y - sigma * y
    _, X, m = lanczos(apply, H.shape[0], nev, v0, dtype=H.dtype, **kw)
    X = X / np.linalg.norm(X, axis=0)
    HX = H @ X
    lam = np.real(np.einsum("ij,ij->j", X.conj(), HX))
    order = np.argsort(lam)
    return lam[order], X[:, order], m


def nearest_shift_invert(H, sigma, nev):
    """Library cross-check: ARPACK in shift-invert mode about sigma (scipy)."""
    vals, vecs = spla.eigsh(H.tocsc(), k=nev, sigma=sigma, which="LM")
    order = np.argsort(vals)
    return vals[order], vecs[:, order]


def residual_norms(H, lam, X):
    """||H x - lambda x|| per column."""
    return np.linalg.norm(H @ X - X * lam[None, :], axis=0)
