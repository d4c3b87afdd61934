"""Explicit CSR assembly of the tight-binding Hamiltonian (oracle; test infrastructure).

What is assembled (paper Section I: empirical sp3s*/sp3d5s* tight binding with strain;
Section III-A item 1: the Schrödinger equation on finite k-points, with the potential from
the Poisson solve "updated in the Hamiltonian"):

* onsite: E_s, E_p (x3), E_d (x5), E_s* of the atom's species, plus U_atom (eV) on every
  orbital of that atom (U = -phi for an electron in the electrostatic potential phi);
* spin-orbit (optional): lambda * L.sigma on the p orbitals, (L_k)_ab = -i eps_kab;
  per-atom basis order (spin, orbital), spin up first;
* bonds: Slater–Koster block for the ideal bond direction scaled by (d0/d)^eta with
  d = d0 (1 + strain of the bond slot); spin diagonal; the block couples the A atom (rows)
  to the B atom (columns), its transpose the reverse;
* Bloch phase exp(i k.T) on a bond whose B end is the periodic image shifted by T
  (supercell-periodic gauge), and its conjugate on the reverse element.

Row index: row = o*natoms + atom, o = spin*norb + orbital (orbital-major, atom-minor).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import lattice
from .sk import sk_block, harrison_factor


def _onsite_diag(params, species):
    """Per-atom onsite energies, shape (natoms, norb)."""
    norb = params.basis
    E = params.onsite[species]                      # (natoms, 4): E_s, E_p, E_d, E_s*
    cols = [E[:, 0], E[:, 1], E[:, 1], E[:, 1]]
    if norb == 10:
        cols += [E[:, 2]] * 5
    cols += [E[:, 3]]
    return np.stack(cols, axis=1)


def so_matrix(norb: int) -> np.ndarray:
    """L.sigma on the p orbitals in the (spin, orbital) basis of one atom, 2norb x 2norb."""
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    Lk = -1j * eps                                   # (L_k)_{ab} = -i eps_{kab}
    sig = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], complex)
    M = np.zeros((2 * norb, 2 * norb), complex)
    for kk in range(3):
        for s1 in range(2):
            for s2 in range(2):
                M[s1 * norb + 1:s1 * norb + 4, s2 * norb + 1:s2 * norb + 4] += sig[kk][s1, s2] * Lk[kk]
    return M


def assemble(spec, params, U_atom=None, kvec=None, spin_orbit=False, row_atoms=None,
             bonds=None):
    """CSR H (FP64, or complex128 with spin-orbit or a Bloch phase).

    kvec: Bloch wave vector in 1/nm (applied on directions with periodic flag 2).
    row_atoms: if given, only rows belonging to these atoms are filled (sampling at scale).
    """
    nx, ny, nz = spec.nx, spec.ny, spec.nz
    N = spec.natoms
    norb = params.basis
    nspin = 2 if spin_orbit else 1
    nb = norb * nspin
    nrows = nb * N
    bloch = kvec is not None and any(p == 2 for p in spec.periodic)
    cplx = spin_orbit or bloch
    dtype = complex if cplx else float
    if bonds is None:
        bonds = lattice.find_bonds(nx, ny, nz, spec.periodic)

    keep_row = None
    if row_atoms is not None:
        keep_row = np.zeros(N, bool)
        keep_row[np.asarray(row_atoms)] = True

    R, C, X = [], [], []

    # onsite
    atoms = np.arange(N) if keep_row is None else np.nonzero(keep_row)[0]
    diag = _onsite_diag(params, spec.species[atoms])
    if U_atom is not None:
        diag = diag + np.asarray(U_atom, float)[atoms][:, None]
    for s in range(nspin):
        for o in range(norb):
            R.append((s * norb + o) * N + atoms)
            C.append((s * norb + o) * N + atoms)
            X.append(diag[:, o].astype(dtype))
    if spin_orbit:
        M = so_matrix(norb)
        lam = params.lambda_so[spec.species[atoms]]
        for o1 in range(nb):
            for o2 in range(nb):
                if M[o1, o2] != 0:
                    R.append(o1 * N + atoms)
                    C.append(o2 * N + atoms)
                    X.append(lam * M[o1, o2])

    # bonds
    u = lattice.BOND_DIRS / np.sqrt(3.0)
    ns = params.nspecies
    blocks = np.zeros((ns, ns, 4, norb, norb))
    for s1 in range(ns):
        for s2 in range(ns):
            for k in range(4):
                blocks[s1, s2, k] = sk_block(u[k], params.V[s1, s2], params.V[s2, s1], norb)
    if keep_row is not None:
        # only bonds that touch a requested row
        m = keep_row[bonds.a] | keep_row[bonds.b]
        bonds = lattice.Bonds(bonds.a[m], bonds.b[m], bonds.k[m], bonds.T[m], bonds.slot[m])
    sa = spec.species[bonds.a]
    sb = spec.species[bonds.b]
    f = harrison_factor(1.0 + spec.strain[bonds.slot], params.eta)
    blk = blocks[sa, sb, bonds.k] * f[:, None, None]          # (nbonds, norb, norb)
    if bloch:
        per2 = np.array([p == 2 for p in spec.periodic])
        Tnm = bonds.T * (spec.a_nm / 4.0) * per2
        phase = np.exp(1j * (Tnm @ np.asarray(kvec, float)))
    else:
        phase = np.ones(len(bonds.a))
    for direction in range(2):
        if direction == 0:
            ra, cb, vals = bonds.a, bonds.b, blk * phase[:, None, None]
        else:
            ra, cb, vals = bonds.b, bonds.a, np.swapaxes(blk, 1, 2) * np.conj(phase)[:, None, None]
        if keep_row is not None:
            m = keep_row[ra]
            ra, cb, vals = ra[m], cb[m], vals[m]
        for o1 in range(norb):
            for o2 in range(norb):
                v = vals[:, o1, o2]
                if not np.any(v != 0):
                    continue
                for s in range(nspin):
                    R.append((s * norb + o1) * N + ra)
                    C.append((s * norb + o2) * N + cb)
                    X.append(v.astype(dtype))
    H = sp.coo_matrix((np.concatenate(X), (np.concatenate(R), np.concatenate(C))),
                      shape=(nrows, nrows)).tocsr()
    H.sum_duplicates()
    return H


def hx_rows(spec, params, x, atoms, **kw):
    """(H x) restricted to the rows of the given atoms (all orbitals, spins), as a dict
    row -> value.  Built from only those rows of H, for sampled checks at full size."""
    H = assemble(spec, params, row_atoms=atoms, **kw)
    y = H @ x
    N = spec.natoms
    nb = H.shape[0] // N
    rows = (np.arange(nb)[:, None] * N + np.asarray(atoms)[None, :]).ravel()
    return rows, y[rows]
