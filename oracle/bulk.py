"""Bulk zincblende H(k) and its spectrum folded onto a periodic supercell (oracle; test infrastructure).

A periodic nx*ny*nz block of conventional cells is invariant under the translations of the
FCC lattice, so its spectrum (at supercell wave vector k0) is the union of the two-atom bulk
spectra at k0 + G over the supercell reciprocal vectors G = 2pi/a (n1/nx, n2/ny, n3/nz),
taken modulo the FCC reciprocal lattice: n1 in [0,2nx), n2 in [0,2ny), n3 in [0,nz),
i.e. 4*nx*ny*nz wave vectors.  This is an exact block diagonalisation, used to pin the
supercell assembly and as the reference spectrum of periodic bulk Si.
"""
from __future__ import annotations

import numpy as np

from .sk import sk_block
from .hamiltonian import so_matrix
from .lattice import BOND_DIRS


def _onsite(params, species, spin_orbit):
    norb = params.basis
    Es, Ep, Ed, Ess = params.onsite[species]
    d = [Es, Ep, Ep, Ep] + ([Ed] * 5 if norb == 10 else []) + [Ess]
    D = np.diag(np.array(d, complex))
    if spin_orbit:
        D = np.kron(np.eye(2), D) + params.lambda_so[species] * so_matrix(norb)
    return D


def bulk_hk(params, kvec, a_nm, spin_orbit=False, species=(0, 0)):
    """Two-atom H(k) (atom A at 0, atom B at a/4 (1,1,1)), unstrained, atom gauge."""
    norb = params.basis
    sA, sB = species
    HAB = np.zeros((norb, norb), complex)
    for k in range(4):
        u = BOND_DIRS[k] / np.sqrt(3.0)
        dvec = BOND_DIRS[k] * a_nm / 4.0
        HAB += sk_block(u, params.V[sA, sB], params.V[sB, sA], norb) * np.exp(1j * np.dot(kvec, dvec))
    if spin_orbit:
        HAB = np.kron(np.eye(2), HAB)
    DA = _onsite(params, sA, spin_orbit)
    DB = _onsite(params, sB, spin_orbit)
    return np.block([[DA, HAB], [HAB.conj().T, DB]])


def folded_wavevectors(nx, ny, nz, a_nm, k0=(0.0, 0.0, 0.0)):
    n1, n2, n3 = np.meshgrid(np.arange(2 * nx), np.arange(2 * ny), np.arange(nz), indexing="ij")
    G = np.stack([n1.ravel() / nx, n2.ravel() / ny, n3.ravel() / nz], axis=1) * (2 * np.pi / a_nm)
    return G + np.asarray(k0, float)[None, :]


def folded_spectrum(params, nx, ny, nz, a_nm, spin_orbit=False, k0=(0.0, 0.0, 0.0)):
    """Sorted eigenvalues of the periodic supercell, from 4*nx*ny*nz bulk H(k) blocks."""
    ev = [np.linalg.eigvalsh(bulk_hk(params, kv, a_nm, spin_orbit))
          for kv in folded_wavevectors(nx, ny, nz, a_nm, k0)]
    return np.sort(np.concatenate(ev))
