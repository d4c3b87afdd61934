"""3-D finite-difference Poisson equation (oracle; test infrastructure).

Paper Section III-A item 3: the charge is fed to a finite-difference Poisson solver (OMEN
3-D uses the Aztec linear solver).  Here: -div(eps0 eps_r grad phi) = rho with constant
eps_r, the standard 7-point stencil on a uniform grid, periodic along x and y, phi = 0 at
both z ends.  SI units inside (m, C/m^3, V); lengths are given in nm.

Grid: nx, ny points along the periodic directions (spacing L/n), nz intervals along z with
nz-1 interior unknowns at z_k = k h_z, k = 1..nz-1.  Unknown index ((k-1)*ny + j)*nx + i;
arrays are shaped (nz-1, ny, nx).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

EPS0 = 8.8541878128e-12     # F/m
Q_E = 1.602176634e-19       # C
KB_EV = 8.617333262e-5      # eV/K


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    Lx_nm: float
    Ly_nm: float
    Lz_nm: float
    eps_r: float = 11.7

    @property
    def h_m(self):
        return np.array([self.Lx_nm / self.nx, self.Ly_nm / self.ny, self.Lz_nm / self.nz]) * 1e-9

    @property
    def shape(self):
        return (self.nz - 1, self.ny, self.nx)


def _second_difference(n, periodic):
    if periodic and n == 1:
        return sp.csr_matrix((1, 1))
    main = -2.0 * np.ones(n)
    off = np.ones(n - 1)
    D = sp.diags([off, main, off], [-1, 0, 1], shape=(n, n), format="lil")
    if periodic and n > 1:
        if n == 2:
            D[0, 1] += 1.0
            D[1, 0] += 1.0
        else:
            D[0, n - 1] = 1.0
            D[n - 1, 0] = 1.0
    return D.tocsr()


def laplacian(grid: Grid):
    """The matrix of -div(grad) on the interior unknowns (1/m^2), symmetric positive definite."""
    hx, hy, hz = grid.h_m
    Dx = _second_difference(grid.nx, True) / hx ** 2
    Dy = _second_difference(grid.ny, True) / hy ** 2
    Dz = _second_difference(grid.nz - 1, False) / hz ** 2
    Ix, Iy, Iz = sp.identity(grid.nx), sp.identity(grid.ny), sp.identity(grid.nz - 1)
    L = sp.kron(Iz, sp.kron(Iy, Dx)) + sp.kron(Iz, sp.kron(Dy, Ix)) + sp.kron(Dz, sp.kron(Iy, Ix))
    return (-L).tocsr()


def solve_direct(grid: Grid, rho):
    """phi (V) for charge density rho (C/m^3), sparse direct solve."""
    A = laplacian(grid)
    b = np.asarray(rho, float).ravel() / (EPS0 * grid.eps_r)
    return spla.spsolve(A.tocsc(), b).reshape(grid.shape)


def solve_cg(grid: Grid, rho, phi0=None, rtol=1e-12, maxiter=100000):
    """Plain conjugate gradients (Hestenes & Stiefel 1952) on the same system."""
    A = laplacian(grid)
    b = np.asarray(rho, float).ravel() / (EPS0 * grid.eps_r)
    x = np.zeros_like(b) if phi0 is None else np.asarray(phi0, float).ravel().copy()
    r = b - A @ x
    p = r.copy()
    rr = r @ r
    bnorm = max(np.linalg.norm(b), 1e-300)
    it = 0
    while np.sqrt(rr) > rtol * bnorm and it < maxiter:
        Ap = A @ p
        a = rr / (p @ Ap)
        x += a * p
        r -= a * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x.reshape(grid.shape), it
