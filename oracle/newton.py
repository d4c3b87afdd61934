"""Newton–Raphson solution of the nonlinear Poisson equation (oracle; test infrastructure).

Paper Section III-A item 3: the charge is fed to the finite-difference Poisson solver and the
converged potential profile is obtained iteratively by Newton–Raphson's method.  The paper
gives no form of the nonlinearity.  Reading (the predictor of Trellakis et al., J. Appl. Phys.
81, 7880 (1997)): inside one outer Schrödinger–Poisson iteration the eigenstates psi_n and
levels E_n computed in the potential phi_in are frozen, and the electrons respond to a change
of the potential by a local shift of the levels (an electron's energy is -phi, in eV per V):

    n_i(phi) = sum_n W_ni f((E_n - u_i - E_F) / kT),   u_i = (G phi)_i - (G phi_in)_i,

W_ni = g_s w_k sum_orb |psi_n(i, orb)|^2 the electrons state n puts on atom i when full, f the
Fermi function, G the trilinear gather of grid potential to the atoms (charge.gather).  The
nonlinear Poisson equation on the interior unknowns is

    F(phi) = L phi - (rho_D + D (-q n(phi))) / eps = 0,   D = G^T / V_cell (charge.deposit),

with L the 7-point operator of poisson.laplacian and eps = eps0 eps_r.  Its Jacobian is

    J = L + (q / eps) D diag(s) G,   s_i = sum_n W_ni f (1 - f) / kT  (>= 0),

symmetric positive definite, so F has one root.  Each Newton step solves J d = -F directly;
iterations stop when max |d| < tol.  At phi = phi_in the predicted density is the frozen
states' density, so a self-consistent potential is a root.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import expit

from . import charge, poisson

Q_E = poisson.Q_E


def gather_matrix(grid, pos_nm):
    """G: (natoms, interior unknowns) trilinear weights; weights on the grounded planes z = 0
    and z = Lz are dropped (phi = 0 there), exactly as charge.gather does."""
    idx, w = charge.cic_stencil(grid, pos_nm)
    plane = grid.ny * grid.nx
    nn = (grid.nz + 1) * plane
    G = sp.csr_matrix((w.ravel(), (np.repeat(np.arange(len(pos_nm)), 8), idx.ravel())), shape=(len(pos_nm), nn))
    return G[:, plane:nn - plane].tocsr()


def predicted_density(W, E, EF, kT, u):
    """n_i and s_i = dn_i/du_i of the frozen states at local level shifts u (eV)."""
    f = expit(-(np.asarray(E, float)[None, :] - np.asarray(u, float)[:, None] - EF) / kT)
    W = np.asarray(W, float)
    return (W * f).sum(axis=1), (W * f * (1.0 - f) / kT).sum(axis=1)


class Problem:
    """One nonlinear Poisson problem: grid, atoms, frozen states (W [natoms, nstates], E),
    E_F, kT, the potential phi_in the states were computed in, and the donor density."""

    def __init__(self, grid, pos_nm, W, E, EF, kT, phi_in, donor_rho):
        self.grid = grid
        self.G = gather_matrix(grid, pos_nm)
        self.D = (self.G.T / np.prod(grid.h_m)).tocsr()
        self.L = poisson.laplacian(grid)
        self.eps = poisson.EPS0 * grid.eps_r
        self.W, self.E, self.EF, self.kT = np.asarray(W, float), np.asarray(E, float), float(EF), float(kT)
        self.u_in = self.G @ np.asarray(phi_in, float).ravel()
        self.rho_d = np.asarray(donor_rho, float).ravel()

    def density(self, phi):
        return predicted_density(self.W, self.E, self.EF, self.kT, self.G @ np.ravel(phi) - self.u_in)

    def residual(self, phi):
        n, _ = self.density(phi)
        return self.L @ np.ravel(phi) - (self.rho_d + self.D @ (-Q_E * n)) / self.eps

    def jacobian(self, phi):
        _, s = self.density(phi)
        return (self.L + (Q_E / self.eps) * (self.D @ sp.diags(s) @ self.G)).tocsc()


def solve(problem: Problem, phi0, tol=1e-12, max_iter=50):
    """Newton–Raphson from phi0; returns (phi, max |step| per iteration)."""
    phi = np.array(phi0, float).ravel()
    steps = []
    for _ in range(max_iter):
        d = spla.spsolve(problem.jacobian(phi), -problem.residual(phi))
        phi += d
        steps.append(float(np.abs(d).max()))
        if steps[-1] < tol:
            break
    return phi.reshape(problem.grid.shape), steps


def state_weights(V, weight, natoms):
    """W column of each eigenvector (rows atom-major within each orbital block): weight *
    sum_orb |psi(orb * natoms + i)|^2."""
    a = np.abs(np.asarray(V)) ** 2
    return weight * a.reshape(-1, natoms, a.shape[1]).sum(axis=0)
