"""Single-band effective-mass Hamiltonian (oracle; test infrastructure).

Paper Section III-A item 1: the Schrödinger solver of the Schrödinger–Poisson loop works on
either the sp3d5s* tight-binding Hamiltonian or an effective-mass Hamiltonian.  The paper
prints no form for the latter; this is the textbook one:

    [ -(hbar^2/2) div(M^-1 grad) + E_c + U(r) ] psi = E psi,

with a constant diagonal mass tensor M = m0 diag(m_x, m_y, m_z) and the second-order central
difference on a uniform grid of spacings h_d, which gives per axis the hopping energy

    t_d = hbar^2 / (2 m0 m_d h_d^2)

and the matrix elements H_ii = E_c + U_i + 2 (t_x + t_y + t_z), H_ij = -t_d for the two
grid neighbours of i along axis d.  Boundaries per axis:

* hard wall (0): psi = 0 one spacing beyond the first and the last point (the coupling is
  dropped);
* periodic (1): the last point couples to the first;
* Bloch (2): periodic with psi(r + L_d e_d) = exp(i k_d L_d) psi(r), L_d = n_d h_d, so the
  element from the last point to the first carries exp(+i k_d L_d) and its reverse the
  conjugate (the same supercell gauge as the tight-binding Bloch phase).

Point index i = (iz*ny + iy)*nx + ix.  Energies in eV, lengths in nm.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

HBAR = 1.054571817e-34          # J s (CODATA 2018)
M0 = 9.1093837015e-31           # kg
Q_E = 1.602176634e-19           # C
# hbar^2 / (2 m0) in eV nm^2
HBAR2_2M0 = HBAR ** 2 / (2.0 * M0) / Q_E * 1e18


def hopping(spec) -> np.ndarray:
    """t_d = hbar^2 / (2 m0 m_d h_d^2) for d = x, y, z (eV)."""
    h = np.asarray(spec.h_nm, dtype=np.float64)
    m = np.asarray(spec.m_rel, dtype=np.float64)
    return HBAR2_2M0 / (m * h * h)


def assemble(spec) -> sp.csr_matrix:
    """CSR H (FP64, complex128 when an axis is Bloch-periodic)."""
    n = (spec.nx, spec.ny, spec.nz)
    N = spec.nx * spec.ny * spec.nz
    t = hopping(spec)
    bloch = any(p == 2 for p in spec.periodic)
    dtype = np.complex128 if bloch else np.float64
    kvec = np.zeros(3) if spec.kvec is None else np.asarray(spec.kvec, dtype=np.float64)
    iz, iy, ix = np.meshgrid(np.arange(spec.nz), np.arange(spec.ny), np.arange(spec.nx), indexing="ij")
    coord = [ix.ravel(), iy.ravel(), iz.ravel()]
    idx = np.arange(N)

    def index(c):
        return (c[2] * spec.ny + c[1]) * spec.nx + c[0]

    U = np.zeros(N) if spec.U is None else np.asarray(spec.U, dtype=np.float64)
    rows = [idx]
    cols = [idx]
    vals = [(spec.ec_eV + U + 2.0 * t.sum()).astype(dtype)]
    for d in range(3):
        # the coupling from each point to its + neighbour along d, and the reverse element
        c = [a.copy() for a in coord]
        c[d] = coord[d] + 1
        inside = c[d] < n[d]
        wrap = ~inside
        if spec.periodic[d] == 0:
            keep = inside
            phase = np.ones(N, dtype=dtype)
        else:
            keep = np.ones(N, dtype=bool)
            c[d] = np.where(wrap, 0, c[d])
            phase = np.ones(N, dtype=dtype)
            if spec.periodic[d] == 2:
                L = n[d] * spec.h_nm[d]
                phase = np.where(wrap, np.exp(1j * kvec[d] * L), 1.0).astype(dtype)
        src = idx[keep]
        dst = index(c)[keep]
        v = -t[d] * phase[keep]
        rows += [src, dst]
        cols += [dst, src]
        vals += [v, np.conj(v)]
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return H.tocsr()       # duplicates (axes of one or two points) are summed
