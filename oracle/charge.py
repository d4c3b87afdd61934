"""Charge from eigenstates, Fermi level, grid deposit and gather (oracle; test infrastructure).

Paper Section III-A item 2: with a given Fermi level the charge is obtained by filling the
states; when the Fermi level is fixed by charge neutrality, charge and Fermi level are found
together.  Here: Fermi–Dirac occupation f((E - E_F)/kT); electron count
N(E_F) = g_s sum_k w_k sum_n f(E_nk); E_F by bisection on the monotone N(E_F) = N_target;
electrons per atom n_i = g_s sum_k w_k sum_n f_nk sum_orb |psi_nk(i, orb)|^2; cloud-in-cell
(trilinear) deposit of per-atom charge onto grid nodes and the adjoint trilinear gather.
"""
from __future__ import annotations

import numpy as np
from scipy.special import expit


def fermi(E, EF, kT):
    return expit(-(np.asarray(E, float) - EF) / kT)


def electron_count(evals_k, weights, EF, kT, gs):
    return gs * sum(w * fermi(e, EF, kT).sum() for e, w in zip(evals_k, weights))


def fermi_level(evals_k, weights, n_target, kT, gs, tol=1e-13):
    """Bisection for N(E_F) = n_target between the lowest and highest given level (+- 50 kT)."""
    allv = np.concatenate([np.asarray(e, float) for e in evals_k])
    lo, hi = allv.min() - 50 * kT, allv.max() + 50 * kT
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if electron_count(evals_k, weights, mid, kT, gs) < n_target:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def atom_density(psi, occ, natoms):
    """sum_n occ_n sum_o |psi[o*natoms + atom, n]|^2 per atom; psi columns = states."""
    w = (np.abs(psi) ** 2) * np.asarray(occ, float)[None, :]
    per_row = w.sum(axis=1)
    return per_row.reshape(-1, natoms).sum(axis=0)


def cic_stencil(grid, pos_nm):
    """Node indices (into the full (nz+1, ny, nx) node array) and trilinear weights, 8 per atom."""
    pos_nm = np.asarray(pos_nm, float)
    h = np.array([grid.Lx_nm / grid.nx, grid.Ly_nm / grid.ny, grid.Lz_nm / grid.nz])
    t = pos_nm / h[None, :]
    i0 = np.floor(t).astype(int)
    f = t - i0
    idx, wts = [], []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ix = (i0[:, 0] + dx) % grid.nx
                iy = (i0[:, 1] + dy) % grid.ny
                iz = np.clip(i0[:, 2] + dz, 0, grid.nz)
                w = (np.where(dx, f[:, 0], 1 - f[:, 0]) * np.where(dy, f[:, 1], 1 - f[:, 1])
                     * np.where(dz, f[:, 2], 1 - f[:, 2]))
                idx.append((iz * grid.ny + iy) * grid.nx + ix)
                wts.append(w)
    return np.stack(idx, 1), np.stack(wts, 1)


def deposit(grid, pos_nm, q):
    """Per-atom charge q (C) -> charge density (C/m^3) on the interior unknowns."""
    idx, w = cic_stencil(grid, pos_nm)
    nodes = np.zeros((grid.nz + 1) * grid.ny * grid.nx)
    np.add.at(nodes, idx.ravel(), (w * np.asarray(q, float)[:, None]).ravel())
    vol = np.prod(np.array([grid.Lx_nm / grid.nx, grid.Ly_nm / grid.ny, grid.Lz_nm / grid.nz]) * 1e-9)
    return nodes.reshape(grid.nz + 1, grid.ny, grid.nx)[1:-1] / vol


def gather(grid, phi_interior, pos_nm):
    """Trilinear interpolation of phi (boundary nodes at 0 V) to the atom positions."""
    full = np.zeros((grid.nz + 1, grid.ny, grid.nx))
    full[1:-1] = phi_interior
    idx, w = cic_stencil(grid, pos_nm)
    return (full.ravel()[idx] * w).sum(axis=1)
