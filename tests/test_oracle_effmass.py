"""Pins of the effective-mass oracle against closed forms and library routines.

The single-band finite-difference Hamiltonian with a constant potential separates into three
1-D chains whose spectra are textbook: a hard-wall chain of n points has the levels
2t(1 - cos(j pi/(n+1))), j = 1..n; a ring of n points with the Bloch condition
psi(x + L) = exp(i k L) psi(x) has 2t(1 - cos((2 pi j + k L)/n)), j = 0..n-1, with the plane
waves exp(i q x), q = (2 pi j + k L)/L, as eigenvectors.  A potential that varies along z only
leaves x and y separable and reduces z to a symmetric tridiagonal matrix (LAPACK's stev).
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import effmass


def chain_levels(n, t, periodic, kL=0.0):
    if periodic == 0:
        j = np.arange(1, n + 1)
        return 2 * t * (1 - np.cos(j * np.pi / (n + 1)))
    j = np.arange(n)
    return 2 * t * (1 - np.cos((2 * np.pi * j + kL) / n))


def separable_levels(spec, U0=0.0):
    t = effmass.hopping(spec)
    n = (spec.nx, spec.ny, spec.nz)
    k = (0, 0, 0) if spec.kvec is None else spec.kvec
    per = [chain_levels(n[d], t[d], spec.periodic[d], k[d] * n[d] * spec.h_nm[d]) for d in range(3)]
    return np.sort([spec.ec_eV + U0 + a + b + c for a, b, c in itertools.product(*per)])


def test_hbar2_over_2m0_is_the_textbook_value():
    # hbar^2/(2 m0) = 3.80998 eV A^2 = 0.0380998 eV nm^2
    assert abs(effmass.HBAR2_2M0 - 0.0380998) < 2e-7


@pytest.mark.parametrize("n,periodic", [((4, 3, 5), (0, 0, 0)), ((4, 3, 5), (1, 1, 0)), ((1, 2, 6), (1, 1, 0)),
                                        ((3, 1, 2), (0, 1, 1))])
def test_constant_potential_box_matches_chain_levels(n, periodic):
    spec = synth.effmass_spec(*n, periodic=periodic, h_nm=(0.21, 0.17, 0.25), m_rel=(0.19, 0.31, 0.916),
                              ec_eV=0.37, u_amp=0.0)
    spec.U = np.full(spec.npoints, -0.05)
    H = effmass.assemble(spec).toarray()
    assert np.array_equal(H, H.conj().T)
    np.testing.assert_allclose(np.linalg.eigvalsh(H), separable_levels(spec, -0.05), atol=1e-12, rtol=0)


@pytest.mark.parametrize("n", [(5, 4, 3), (1, 2, 3), (2, 1, 4)])
def test_bloch_box_matches_shifted_ring_levels(n):
    kvec = (0.7, -1.3, 0.4)
    spec = synth.effmass_spec(*n, periodic=(2, 2, 2), h_nm=(0.2, 0.23, 0.19), kvec=kvec, ec_eV=0.1, u_amp=0.0)
    H = effmass.assemble(spec).toarray()
    assert H.dtype == np.complex128
    np.testing.assert_allclose(H, H.conj().T, atol=0, rtol=0)
    np.testing.assert_allclose(np.linalg.eigvalsh(H), separable_levels(spec), atol=1e-12, rtol=0)


def test_bloch_plane_waves_are_eigenvectors():
    """The sign of the wrap phase: exp(i q x) with q = (2 pi j + k L)/L satisfies the Bloch
    condition only with exp(+i k L) on the element from the last point to the first."""
    n, h, kx = 7, 0.2, 2.1
    spec = synth.effmass_spec(n, 1, 1, periodic=(2, 0, 0), h_nm=(h, 0.2, 0.2), kvec=(kx, 0, 0), u_amp=0.0)
    H = effmass.assemble(spec).toarray()
    t = effmass.hopping(spec)
    L = n * h
    x = np.arange(n) * h
    for j in range(n):
        q = (2 * np.pi * j + kx * L) / L
        psi = np.exp(1j * q * x)
        e = 2 * t[0] * (1 - np.cos(q * h)) + 2 * (t[1] + t[2])
        assert np.abs(H @ psi - e * psi).max() < 1e-12


def test_k_shift_by_a_reciprocal_vector_is_a_gauge():
    spec0 = synth.effmass_spec(4, 3, 2, periodic=(2, 2, 0), u_amp=0.05, seed=3, kvec=(0.0, 0.0, 0.0))
    L = (4 * 0.2, 3 * 0.2)
    spec1 = synth.effmass_spec(4, 3, 2, periodic=(2, 2, 0), u_amp=0.05, seed=3,
                               kvec=(2 * np.pi / L[0], -2 * np.pi / L[1], 0.0))
    w0 = np.linalg.eigvalsh(effmass.assemble(spec0).toarray())
    w1 = np.linalg.eigvalsh(effmass.assemble(spec1).toarray())
    np.testing.assert_allclose(w1, w0, atol=1e-12, rtol=0)


def test_potential_along_z_reduces_to_a_tridiagonal_solve():
    nx, ny, nz = 3, 4, 9
    spec = synth.effmass_spec(nx, ny, nz, periodic=(1, 1, 0), h_nm=(0.2, 0.2, 0.3), ec_eV=0.2, u_amp=0.0)
    Uz = synth.rng(11, 99).uniform(-0.3, 0.3, size=nz)
    spec.U = np.repeat(Uz, nx * ny)                  # U depends on iz only
    t = effmass.hopping(spec)
    mu = sla.eigh_tridiagonal(spec.ec_eV + Uz + 2 * t[2], np.full(nz - 1, -t[2]), eigvals_only=True)
    ex = chain_levels(nx, t[0], 1)
    ey = chain_levels(ny, t[1], 1)
    ref = np.sort([a + b + c for a, b, c in itertools.product(ex, ey, mu)])
    w = np.linalg.eigvalsh(effmass.assemble(spec).toarray())
    np.testing.assert_allclose(w, ref, atol=1e-12, rtol=0)


def test_random_potential_sits_on_the_diagonal_in_point_order():
    """Without hopping partners (one point per axis, hard walls) H is diagonal: E_c + U_i + 2 sum t."""
    spec = synth.effmass_spec(1, 1, 1, seed=4, ec_eV=0.3)
    H = effmass.assemble(spec).toarray()
    assert H.shape == (1, 1)
    assert abs(H[0, 0] - (0.3 + spec.U[0] + 2 * effmass.hopping(spec).sum())) < 1e-15
    # first-order perturbation theory: d E_j / d U_i = |psi_j(i)|^2 (Hellmann–Feynman)
    spec = synth.effmass_spec(3, 2, 4, seed=5, periodic=(0, 1, 0))
    H0 = effmass.assemble(spec).toarray()
    w, V = np.linalg.eigh(H0)
    i, eps = 13, 1e-6
    spec.U = spec.U.copy()
    spec.U[i] += eps
    w1 = np.linalg.eigvalsh(effmass.assemble(spec).toarray())
    np.testing.assert_allclose((w1 - w) / eps, np.abs(V[i, :]) ** 2, atol=1e-6, rtol=0)


def test_continuum_limit_of_the_ground_state():
    """Hard-wall box of side L: the lowest level tends to sum_d hbar^2 pi^2 / (2 m0 m_d L_d^2)
    with an O(h^2) discretisation error."""
    L, m = np.array([4.0, 5.0, 6.0]), np.array([0.19, 0.19, 0.916])
    exact = effmass.HBAR2_2M0 * np.pi ** 2 * np.sum(1.0 / (m * L * L))
    errs = []
    for n in (10, 20):
        h = L / (n + 1)
        spec = synth.effmass_spec(n, n, n, h_nm=tuple(h), m_rel=tuple(m), u_amp=0.0)
        e0 = separable_levels(spec)[0]
        H = effmass.assemble(spec)
        import scipy.sparse.linalg as spla
        w = spla.eigsh(H, k=1, sigma=0.0, return_eigenvectors=False)
        assert abs(w[0] - e0) < 1e-10
        errs.append(abs(e0 - exact))
    assert errs[1] < errs[0] / 3.5          # second-order convergence
