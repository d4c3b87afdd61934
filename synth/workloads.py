"""Seeded synthetic workloads (random draws and input layouts only).

Layouts (the C-ABI uses the same ones):

* Conventional zincblende cell = 8 sites.  Site b in 0..3 is on the first FCC sublattice
  ("A"), b in 4..7 on the second ("B" = A site + a/4 (1,1,1)).
* cell = (iz*ny + iy)*nx + ix;  atom = b*ncells + cell  (sublattice-major, cell-minor).
* Bond slot of A site s (0..3) in cell c along direction k (0..3):
  slot = (k*4 + s)*ncells + c, 16*ncells slots.  Directions in units of a/4:
  k=0 (1,1,1), k=1 (1,-1,-1), k=2 (-1,1,-1), k=3 (-1,-1,1), from the A atom to the B atom.
* Two-centre parameter order (14): ss_sigma, s*s*_sigma, ss*_sigma, sp_sigma, s*p_sigma,
  sd_sigma, s*d_sigma, pp_sigma, pp_pi, pd_sigma, pd_pi, dd_sigma, dd_pi, dd_delta.
  V[i, j, p] is the integral with the first-named orbital on an atom of species i and the
  second on an atom of species j.
* Onsite parameter order (4): E_s, E_p, E_d, E_s*.

Random streams: a SeedSequence keyed by (seed, stream) per draw kind.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

STREAM_TB, STREAM_SPECIES, STREAM_STRAIN, STREAM_SIGMA, STREAM_DONOR, STREAM_START, STREAM_DOPING = range(7)

PARAM_NAMES = ("ss_sigma", "s*s*_sigma", "ss*_sigma", "sp_sigma", "s*p_sigma", "sd_sigma",
               "s*d_sigma", "pp_sigma", "pp_pi", "pd_sigma", "pd_pi", "dd_sigma", "dd_pi",
               "dd_delta")
SP3S_PARAMS = (0, 1, 2, 3, 4, 7, 8)           # the seven sp3s* two-centre integrals
ONSITE_NAMES = ("E_s", "E_p", "E_d", "E_s*")

SP3S, SP3D5S = 5, 10                          # orbitals per atom and spin
SI_A_NM = 0.5431                              # silicon lattice constant (nm)


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream)]))


@dataclass
class TBParams:
    """Tight-binding parameter tables (eV) in the C-ABI layout."""
    basis: int                                # SP3S (5) or SP3D5S (10)
    onsite: np.ndarray                        # (nspecies, 4)
    V: np.ndarray                             # (nspecies, nspecies, 14)
    lambda_so: np.ndarray                     # (nspecies,)
    eta: float = 2.0                          # Harrison exponent, V(d) = V(d0) (d0/d)^eta

    @property
    def nspecies(self) -> int:
        return self.onsite.shape[0]


def draw_tb_params(seed: int, basis: int, nspecies: int = 1,
                   so_range=(0.01, 0.3)) -> TBParams:
    """Per-species draws; pairs of unlike species take the mean of the two like-pair sets.

    Ranges: E_s [-6,-3], E_p [0,3], E_d [3,6], E_s* [5,8]; every two-centre integral in
    [-3,3]; lambda_SO in so_range.  sp3s* leaves the d entries at zero.
    """
    g = rng(seed, STREAM_TB)
    onsite = np.zeros((nspecies, 4))
    own = np.zeros((nspecies, 14))
    lam = np.zeros(nspecies)
    for s in range(nspecies):
        onsite[s] = [g.uniform(-6, -3), g.uniform(0, 3), g.uniform(3, 6), g.uniform(5, 8)]
        own[s] = g.uniform(-3, 3, size=14)
        lam[s] = g.uniform(*so_range)
    if basis == SP3S:
        onsite[:, 2] = 0.0
        mask = np.zeros(14, bool)
        mask[list(SP3S_PARAMS)] = True
        own[:, ~mask] = 0.0
    V = 0.5 * (own[:, None, :] + own[None, :, :])
    return TBParams(basis=basis, onsite=onsite, V=V, lambda_so=lam)


@dataclass
class LatticeSpec:
    """A zincblende block of nx*ny*nz conventional cells with per-site species and per-bond strain.

    periodic[d]: 0 hard wall (bonds leaving the block are dropped), 1 periodic, 2 periodic
    with a Bloch phase (k given at assembly).
    """
    nx: int
    ny: int
    nz: int
    periodic: tuple
    species: np.ndarray                       # uint8 [8*ncells]
    strain: np.ndarray                        # float64 [16*ncells], relative bond-length change
    a_nm: float = SI_A_NM

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def natoms(self) -> int:
        return 8 * self.ncells


def lattice_spec(nx: int, ny: int, nz: int, periodic=(1, 1, 1), seed: int = 0,
                 alloy_fraction: float = 0.0, strain_amp: float = 0.0,
                 a_nm: float = SI_A_NM) -> LatticeSpec:
    """Species 1 with probability alloy_fraction per site (stream 1); strain U[-amp, amp] (stream 2)."""
    ncells = nx * ny * nz
    if alloy_fraction > 0:
        species = (rng(seed, STREAM_SPECIES).random(8 * ncells) < alloy_fraction).astype(np.uint8)
    else:
        species = np.zeros(8 * ncells, np.uint8)
    if strain_amp > 0:
        strain = rng(seed, STREAM_STRAIN).uniform(-strain_amp, strain_amp, size=16 * ncells)
    else:
        strain = np.zeros(16 * ncells)
    return LatticeSpec(nx, ny, nz, tuple(int(p) for p in periodic), species, strain, a_nm)


def start_block(seed: int, n: int, b: int = 1, dtype=np.float64) -> np.ndarray:
    """Lanczos start block, uniform [-1,1] (stream 5), shape (b, n) (row = one vector)."""
    g = rng(seed, STREAM_START)
    x = g.uniform(-1, 1, size=(b, n))
    if np.issubdtype(np.dtype(dtype), np.complexfloating):
        x = x + 1j * g.uniform(-1, 1, size=(b, n))
    return x.astype(dtype)


def sigma_offset_fraction(seed: int) -> float:
    """u ~ U[-0.05, 0.05] (stream 3); the shift is sigma = centre + u * width."""
    return float(rng(seed, STREAM_SIGMA).uniform(-0.05, 0.05))


def random_vectors(seed: int, n: int, b: int = 1, dtype=np.float64, stream: int = 99) -> np.ndarray:
    """Generic uniform [-1,1] test vectors, shape (b, n)."""
    g = rng(seed, stream)
    x = g.uniform(-1, 1, size=(b, n))
    if np.issubdtype(np.dtype(dtype), np.complexfloating):
        x = x + 1j * g.uniform(-1, 1, size=(b, n))
    return x.astype(dtype)


# Named workloads -------------------------------------------------------------------------

def config_si_periodic(n: int = 8, seed: int = 1):
    """Bulk Si, n^3 cells, fully periodic, sp3s*, one species, unstrained (4,096 atoms at n=8)."""
    return lattice_spec(n, n, n, (1, 1, 1), seed), draw_tb_params(seed, SP3S, 1)


def config_sige_alloy(n: int = 50, seed: int = 2, spin_orbit: bool = False):
    """Si0.7Ge0.3 random alloy, n^3 cells, hard walls, bond strain U[-2%,2%], sp3d5s*
    (1,000,000 atoms at n=50)."""
    lat = lattice_spec(n, n, n, (0, 0, 0), seed, alloy_fraction=0.3, strain_amp=0.02)
    return lat, draw_tb_params(seed, SP3D5S, 2)


# Delta-doped Si ------------------------------------------------------------------------------
# First seeded sp3d5s* Si draw with a bulk gap >= 0.5 eV, found by
# tests/golden/make_gapped_si_params.py (stored in tests/golden/gapped_si_params.json).
GAPPED_SI_SEED = 163
GAPPED_SI_EV, GAPPED_SI_EC = -2.627017511981574, -1.6808215901542354
Q_E = 1.602176634e-19


def gapped_si_params() -> TBParams:
    return draw_tb_params(GAPPED_SI_SEED, SP3D5S, 1)


def draw_doping(seed: int, ns_range=(1e13, 2e14), w_range=(0.5, 2.0)):
    """Sheet density N_s (cm^-2, log-uniform) and FWHM w (nm, uniform), stream 6."""
    g = rng(seed, STREAM_DOPING)
    ns = 10 ** g.uniform(np.log10(ns_range[0]), np.log10(ns_range[1]))
    w = g.uniform(*w_range)
    return float(ns), float(w)


def donor_rho_on_grid(ns_cm2, fwhm_nm, nx, ny, nz, Lz_nm, z0_nm=None):
    """Laterally uniform Gaussian sheet of ionised donors, charge density (C/m^3) on the
    interior grid planes z_k = k Lz/nz, k = 1..nz-1, normalised so that sum_k rho_k h_z equals
    e N_s exactly (shape (nz-1, ny, nx))."""
    z0 = 0.5 * Lz_nm if z0_nm is None else z0_nm
    hz = Lz_nm / nz
    z = np.arange(1, nz) * hz
    s = fwhm_nm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    prof = np.exp(-0.5 * ((z - z0) / s) ** 2)
    prof /= prof.sum() * hz * 1e-9                       # 1/m
    rho_z = Q_E * ns_cm2 * 1e4 * prof                    # C/m^3
    return np.broadcast_to(rho_z[:, None, None], (nz - 1, ny, nx)).copy()


def delta_layer(nxy: int, nz_cells: int, seed: int = 5):
    """Si slab of nxy x nxy x nz_cells cells, periodic with a Bloch phase in x and y, hard walls
    in z, gapped sp3d5s* Si parameters; returns (spec, params, (N_s, w))."""
    spec = lattice_spec(nxy, nxy, nz_cells, (2, 2, 0), seed)
    return spec, gapped_si_params(), draw_doping(seed)


def donor_sheet_potential(spec: LatticeSpec, seed: int, lam_tf_nm: float, eps_r: float = 11.7,
                          frac: float = 0.25):
    """Onsite potential energy (eV per atom) of a seeded donor sheet: a fraction `frac` of the
    atoms of the (001) atomic plane nearest mid-z (stream 4) carry +e, screened Coulomb
    U(r) = -(e^2 / (4 pi eps0 eps_r r)) exp(-r / lam_TF), summed over the donors and their
    lateral periodic images with r <= 8 lam_TF; r is clamped at the bond length a sqrt(3)/4."""
    g = rng(seed, STREAM_DONOR)
    a = spec.a_nm
    iz, iy, ix = np.meshgrid(np.arange(spec.nz), np.arange(spec.ny), np.arange(spec.nx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1) * 4
    sites = np.array([[0, 0, 0], [0, 2, 2], [2, 0, 2], [2, 2, 0], [1, 1, 1], [1, 3, 3], [3, 1, 3], [3, 3, 1]])
    pos = ((sites[:, None, :] + cells[None, :, :]).reshape(-1, 3)) * (a / 4.0)
    zmid = 0.5 * spec.nz * a
    zs = np.unique(pos[:, 2])
    zplane = zs[np.argmin(np.abs(zs - zmid))]
    plane = np.nonzero(np.abs(pos[:, 2] - zplane) < 1e-9)[0]
    nd = max(1, int(round(frac * len(plane))))
    donors = pos[g.choice(plane, size=nd, replace=False)]
    Lx, Ly = spec.nx * a, spec.ny * a
    rc = 8.0 * lam_tf_nm
    nix, niy = int(np.ceil(rc / Lx)) + 1, int(np.ceil(rc / Ly)) + 1
    coul = 1.439964547 / eps_r           # e^2 / (4 pi eps0) in eV nm, screened by eps_r
    rmin = a * np.sqrt(3.0) / 4.0
    U = np.zeros(len(pos))
    for sx in range(-nix, nix + 1):
        for sy in range(-niy, niy + 1):
            img = donors + np.array([sx * Lx, sy * Ly, 0.0])
            for d in img:
                r = np.linalg.norm(pos - d[None, :], axis=1)
                m = r <= rc
                rr = np.maximum(r[m], rmin)
                U[m] -= coul * np.exp(-rr / lam_tf_nm) / rr
    return U


def draw_kbatch_instances(seed: int, n_instances: int = 8, sizes=(2, 3, 4, 6, 8), nz: int = 80):
    """Instance lateral sizes (stream 1) and Thomas–Fermi lengths U[1, 5] nm (stream 4)."""
    g = rng(seed, STREAM_SPECIES)
    lat_sizes = [int(g.choice(sizes)) for _ in range(n_instances)]
    lam = rng(seed + 1000, STREAM_DONOR).uniform(1.0, 5.0, size=n_instances)
    return [(s, nz, float(l)) for s, l in zip(lat_sizes, lam)]


def mlp_init(seed: int, sizes=(256, 512, 512, 256)) -> np.ndarray:
    """Glorot-uniform weights, zero biases, flat FP32 in the C-ABI layout (stream 7)."""
    g = rng(seed, 7)
    parts = []
    for l in range(3):
        fan_in, fan_out = sizes[l], sizes[l + 1]
        a = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(g.uniform(-a, a, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


# Effective-mass grids ------------------------------------------------------------------------

STREAM_EFFMASS = 8
SI_M_LONG, SI_M_TRANS = 0.916, 0.19          # Si conduction-band valley masses (units of m0)


@dataclass
class EffMassSpec:
    """Uniform nx x ny x nz grid for the single-band effective-mass Hamiltonian.  Point index
    i = (iz*ny + iy)*nx + ix; U (eV per point, flat in that order) or None."""
    nx: int
    ny: int
    nz: int
    h_nm: tuple = (0.2, 0.2, 0.2)
    m_rel: tuple = (SI_M_TRANS, SI_M_TRANS, SI_M_LONG)
    periodic: tuple = (0, 0, 0)
    ec_eV: float = 0.0
    kvec: tuple = None
    U: np.ndarray = None

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz


def effmass_spec(nx: int, ny: int, nz: int, seed: int = 0, periodic=(0, 0, 0), h_nm=(0.2, 0.2, 0.2),
                 m_rel=(SI_M_TRANS, SI_M_TRANS, SI_M_LONG), ec_eV: float = 0.0, kvec=None,
                 u_amp: float = 0.1) -> EffMassSpec:
    """A grid with a seeded random potential U ~ U[-u_amp, u_amp] eV per point (stream 8)."""
    U = rng(seed, STREAM_EFFMASS).uniform(-u_amp, u_amp, size=nx * ny * nz) if u_amp > 0 else None
    return EffMassSpec(nx, ny, nz, tuple(h_nm), tuple(m_rel), tuple(periodic), ec_eV,
                       None if kvec is None else tuple(kvec), U)


# Valence-force-field parameters ----------------------------------------------------------------

STREAM_VFF = 9
GE_A_NM = 0.5658                              # germanium lattice constant (nm)
N_PER_M_IN_EV_PER_NM2 = 1.0 / 1.602176634e-19 * 1e-18   # 1 N/m = 6.2415 eV/nm^2


@dataclass
class VFFParams:
    """Keating force constants per species: natural lattice constant a (nm), bond stretching
    alpha and bond bending beta (eV/nm^2)."""
    a_nm: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray


def draw_vff_params(seed: int, nspecies: int = 2) -> VFFParams:
    """Species 0 at the Si lattice constant, species 1 at Ge's; alpha ~ U[38, 50] N/m and
    beta ~ U[10, 15] N/m per species (stream 9)."""
    g = rng(seed, STREAM_VFF)
    a = np.array([SI_A_NM, GE_A_NM, SI_A_NM, GE_A_NM][:nspecies])
    alpha = g.uniform(38.0, 50.0, size=nspecies) * N_PER_M_IN_EV_PER_NM2
    beta = g.uniform(10.0, 15.0, size=nspecies) * N_PER_M_IN_EV_PER_NM2
    return VFFParams(a, alpha, beta)
