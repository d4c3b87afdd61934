"""Slater–Koster two-centre bond blocks (oracle; test infrastructure).

Definition followed (Slater & Koster, Phys. Rev. 94, 1498 (1954)): in a frame whose z axis
points from atom 1 to atom 2, the two-centre integrals are diagonal in the magnetic quantum
number about the bond axis; their nonzero values are the sigma/pi/delta parameters.  The
block for any bond direction is that bond-frame block expressed in the global orbitals by
rotation.  Harrison scaling multiplies every two-centre integral by (d0/d)^eta.  The paper
(Section I and abstract) names the sp3s* and sp3d5s* models and strain but prints no formula;
these are the standard definitions it relies on.

Orbital order per atom: s, px, py, pz, [dyz, dzx, dxy, dx2-y2, d3z2-r2], s*.
Real d orbitals on the unit sphere: sqrt3*yz, sqrt3*zx, sqrt3*xy, (sqrt3/2)(x^2-y^2),
z^2-(x^2+y^2)/2 (all with equal norm).

Parameter index (14): ss_sigma, s*s*_sigma, ss*_sigma, sp_sigma, s*p_sigma, sd_sigma,
s*d_sigma, pp_sigma, pp_pi, pd_sigma, pd_pi, dd_sigma, dd_pi, dd_delta.  V12 holds the
integrals with the first-named orbital on atom 1, V21 with it on atom 2.
"""
from __future__ import annotations

import numpy as np

SS, SSSTAR_SS, SSS, SP, SSP, SD, SSD, PPS, PPP, PDS, PDP, DDS, DDP, DDD = range(14)
S3 = np.sqrt(3.0)


def _orbital_layout(basis: int):
    """(index of s, slice of p, slice of d or None, index of s*)."""
    if basis == 5:
        return 0, slice(1, 4), None, 4
    if basis == 10:
        return 0, slice(1, 4), slice(4, 9), 9
    raise ValueError("basis must be 5 (sp3s*) or 10 (sp3d5s*)")


def _d_quadratic_forms():
    """Traceless symmetric Q_a with f_a(r) = r^T Q_a r for the five real d orbitals."""
    Q = np.zeros((5, 3, 3))
    h = S3 / 2
    Q[0][1, 2] = Q[0][2, 1] = h           # sqrt3 * y z
    Q[1][2, 0] = Q[1][0, 2] = h           # sqrt3 * z x
    Q[2][0, 1] = Q[2][1, 0] = h           # sqrt3 * x y
    Q[3] = np.diag([h, -h, 0.0])          # (sqrt3/2)(x^2 - y^2)
    Q[4] = np.diag([-0.5, -0.5, 1.0])     # z^2 - (x^2+y^2)/2
    return Q


_QD = _d_quadratic_forms()


def orbital_rotation(R: np.ndarray, basis: int) -> np.ndarray:
    """D with f_a(R r) = sum_a' D[a', a] f_a'(r) for the orbital functions of one atom."""
    D = np.zeros((basis, basis))
    s, p, d, ss = _orbital_layout(basis)
    D[s, s] = 1.0
    D[ss, ss] = 1.0
    D[p, p] = R.T                          # f_i(R r) = sum_j R_ij r_j
    if d is not None:
        RQR = np.einsum("ji,ajk,kl->ail", R, _QD, R)     # R^T Q_a R
        norm = np.einsum("aij,aij->a", _QD, _QD)
        D[d, d] = np.einsum("bij,aij->ba", _QD, RQR) / norm[:, None]
    return D


def bond_frame_block(V12: np.ndarray, V21: np.ndarray, basis: int) -> np.ndarray:
    """Block <1 a|H|2 b> for atom 2 on the +z axis of atom 1 (the definition of sigma/pi/delta).

    An orbital on atom 1 whose lobe along +z is odd picks up the sign (-1)^l of inversion
    when the parameter is named with the other atom's orbital first (V21).
    """
    B = np.zeros((basis, basis))
    s, p, d, ss = _orbital_layout(basis)
    px, py, pz = p.start, p.start + 1, p.start + 2
    # s-like pairs
    B[s, s] = V12[SS]
    B[ss, ss] = V12[SSSTAR_SS]
    B[s, ss] = V12[SSS]
    B[ss, s] = V21[SSS]
    # s - p (sigma only, along z)
    B[s, pz] = V12[SP]
    B[ss, pz] = V12[SSP]
    B[pz, s] = -V21[SP]
    B[pz, ss] = -V21[SSP]
    # p - p
    B[pz, pz] = V12[PPS]
    B[px, px] = V12[PPP]
    B[py, py] = V12[PPP]
    if d is not None:
        dyz, dzx, dxy, dx2, dz2 = range(d.start, d.stop)
        B[s, dz2] = V12[SD]
        B[ss, dz2] = V12[SSD]
        B[dz2, s] = V21[SD]
        B[dz2, ss] = V21[SSD]
        B[pz, dz2] = V12[PDS]
        B[px, dzx] = V12[PDP]
        B[py, dyz] = V12[PDP]
        B[dz2, pz] = -V21[PDS]
        B[dzx, px] = -V21[PDP]
        B[dyz, py] = -V21[PDP]
        B[dz2, dz2] = V12[DDS]
        B[dzx, dzx] = V12[DDP]
        B[dyz, dyz] = V12[DDP]
        B[dxy, dxy] = V12[DDD]
        B[dx2, dx2] = V12[DDD]
    return B


def frame_to(u: np.ndarray) -> np.ndarray:
    """A rotation R (columns e1, e2, u) with R e_z = u."""
    u = np.asarray(u, float) / np.linalg.norm(u)
    t = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = t - u * (t @ u)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    return np.stack([e1, e2, u], axis=1)


def sk_block(u, V12, V21, basis: int) -> np.ndarray:
    """<atom1 a|H|atom2 b> for the unit vector u from atom 1 to atom 2 (global orbitals)."""
    R = frame_to(u)
    D = orbital_rotation(R, basis)
    return D.T @ bond_frame_block(np.asarray(V12, float), np.asarray(V21, float), basis) @ D


def harrison_factor(d_over_d0, eta: float = 2.0):
    """Harrison scaling of two-centre integrals with bond length: (d0/d)^eta."""
    return np.asarray(d_over_d0, float) ** (-eta)
