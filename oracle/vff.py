"""Keating valence force field: strain energy, forces and relaxation (oracle; test infrastructure).

Paper Section II-B (strain test): NEMO/OMEN 3-D relax the atom positions of a structure by
minimising the total strain energy of an atomistic valence force field (VFF) before the
electronic-structure step.  The paper prints no form; this is Keating's (Phys. Rev. 145, 637
(1966)), written per bond and per bond angle:

    E = sum_bonds  3 alpha_b / (8 d_b^2) (r_b.r_b - d_b^2)^2
      + sum_atoms sum_{bond pairs p<q at the atom}  3 beta_pq / (8 d_p d_q) (r_p.r_q + d_p d_q / 3)^2

r_p is the vector from the atom to its neighbour along bond p; d_b the natural bond length of
the bond's species pair (sqrt(3)/4 of the species' lattice constant; the mean for a mixed
pair); alpha_b the mean of the two species' bond-stretching constants; beta_pq the mean of the
bond-bending constants of the two bonds.  Atom positions are x = F x0 + u: x0 the ideal
zincblende positions at the structure's lattice constant, F a fixed homogeneous deformation of
the whole box (periodic images move with it), u the displacements that the relaxation finds.
Bonds leaving a hard wall are absent (free surfaces, no passivation).

Units: nm, eV; alpha, beta in eV/nm^2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.optimize as so

from . import lattice


@dataclass
class Geometry:
    x0: np.ndarray        # (natoms, 3) ideal positions (nm)
    bonds: lattice.Bonds
    bvec0: np.ndarray     # (nbonds, 3) ideal A->B bond vectors (nm), image shift included
    d: np.ndarray         # (nbonds,) natural bond length of the pair
    alpha: np.ndarray     # (nbonds,)
    beta: np.ndarray      # (nbonds,)
    # angles: bond indices p, q and the signs that turn the A->B vectors into vectors leaving
    # the vertex atom (+1 at an A vertex, -1 at a B vertex)
    p: np.ndarray
    q: np.ndarray
    sgn: np.ndarray


def geometry(spec, vp) -> Geometry:
    bonds = lattice.find_bonds(spec.nx, spec.ny, spec.nz, spec.periodic)
    q4 = spec.a_nm / 4.0
    x0 = lattice.positions(spec.nx, spec.ny, spec.nz) * q4
    bvec0 = lattice.BOND_DIRS[bonds.k] * q4
    sa = spec.species[bonds.a].astype(int)
    sb = spec.species[bonds.b].astype(int)
    dnat = np.sqrt(3.0) / 4.0 * np.asarray(vp.a_nm)
    d = 0.5 * (dnat[sa] + dnat[sb])
    alpha = 0.5 * (np.asarray(vp.alpha)[sa] + np.asarray(vp.alpha)[sb])
    beta = 0.5 * (np.asarray(vp.beta)[sa] + np.asarray(vp.beta)[sb])
    # bonds meeting at each atom: at its A end (+) or its B end (-)
    natoms = spec.natoms
    ends = [[] for _ in range(natoms)]
    for j in range(len(bonds.a)):
        ends[bonds.a[j]].append((j, 1.0))
        ends[bonds.b[j]].append((j, -1.0))
    P, Q, S = [], [], []
    for lst in ends:
        for u in range(len(lst)):
            for v in range(u + 1, len(lst)):
                P.append(lst[u][0])
                Q.append(lst[v][0])
                S.append(lst[u][1] * lst[v][1])
    return Geometry(x0, bonds, bvec0, d, alpha, beta, np.array(P, int), np.array(Q, int), np.array(S))


def bond_vectors(g: Geometry, u: np.ndarray, F=None) -> np.ndarray:
    """A->B bond vectors F r0 + u_B - u_A (nm)."""
    F = np.eye(3) if F is None else np.asarray(F, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64).reshape(-1, 3)
    return g.bvec0 @ F.T + u[g.bonds.b] - u[g.bonds.a]


def energy(g: Geometry, u: np.ndarray, F=None) -> float:
    r = bond_vectors(g, u, F)
    rr = np.einsum("ij,ij->i", r, r)
    e_bond = np.sum(3.0 * g.alpha / (8.0 * g.d ** 2) * (rr - g.d ** 2) ** 2)
    dd = g.d[g.p] * g.d[g.q]
    c = g.sgn * np.einsum("ij,ij->i", r[g.p], r[g.q]) + dd / 3.0
    bpq = 0.5 * (g.beta[g.p] + g.beta[g.q])
    e_ang = np.sum(3.0 * bpq / (8.0 * dd) * c ** 2)
    return float(e_bond + e_ang)


def gradient(g: Geometry, u: np.ndarray, F=None) -> np.ndarray:
    """dE/du, shape (natoms, 3)."""
    r = bond_vectors(g, u, F)
    rr = np.einsum("ij,ij->i", r, r)
    # dE/dr per bond
    gr = (3.0 * g.alpha / (2.0 * g.d ** 2) * (rr - g.d ** 2))[:, None] * r
    dd = g.d[g.p] * g.d[g.q]
    c = g.sgn * np.einsum("ij,ij->i", r[g.p], r[g.q]) + dd / 3.0
    bpq = 0.5 * (g.beta[g.p] + g.beta[g.q])
    w = (3.0 * bpq / (4.0 * dd) * c * g.sgn)[:, None]
    np.add.at(gr, g.p, w * r[g.q])
    np.add.at(gr, g.q, w * r[g.p])
    # r = ... + u_B - u_A
    out = np.zeros((g.x0.shape[0], 3))
    np.add.at(out, g.bonds.b, gr)
    np.subtract.at(out, g.bonds.a, gr)
    return out


def relax(g: Geometry, F=None, u0=None, gtol=1e-10, maxiter=20000):
    """Displacements minimising E at fixed box deformation F.  Returns (u, E, max |force|).

    scipy's L-BFGS descends until the energy itself stops resolving the step (forces near
    1e-7 eV/nm for energies of a few eV); Newton–Krylov on the forces (scipy.optimize.root)
    then drives them to gtol, the forces being computed without that cancellation."""
    n = g.x0.shape[0]
    x = np.zeros(3 * n) if u0 is None else np.asarray(u0, dtype=np.float64).ravel().copy()
    res = so.minimize(lambda v: energy(g, v, F), x, jac=lambda v: gradient(g, v, F).ravel(), method="L-BFGS-B",
                      options={"gtol": gtol, "ftol": 0.0, "maxiter": maxiter, "maxcor": 30})
    x = res.x
    if np.abs(gradient(g, x, F)).max() > gtol:
        x = so.root(lambda v: gradient(g, v, F).ravel(), x, method="krylov", options={"fatol": gtol}).x
    u = x.reshape(n, 3)
    return u, energy(g, u, F), float(np.abs(gradient(g, u, F)).max())


def bond_strain(g: Geometry, u: np.ndarray, F=None, nslots: int = None) -> np.ndarray:
    """Relative bond-length change |r_b| / d_b - 1 per bond slot (the tight-binding assembly's
    strain input: slot (k*4 + s)*ncells + cell of the A atom; slots without a bond are 0)."""
    r = bond_vectors(g, u, F)
    n = 16 * (g.x0.shape[0] // 8) if nslots is None else nslots
    out = np.zeros(n)
    out[g.bonds.slot] = np.sqrt(np.einsum("ij,ij->i", r, r)) / g.d - 1.0
    return out
