"""Pins of the Keating valence-force-field oracle.

Keating's model has published elastic constants (Keating 1966; Martin 1970): with bond
stretching alpha, bond bending beta and lattice constant a,
    C11 = (alpha + 3 beta)/a,   C12 = (alpha - beta)/a,
    C44 = 4 alpha beta / (a (alpha + beta))      (sublattices relaxed under shear),
    C44_0 = (alpha + beta)/a                     (unrelaxed),
and they obey Keating's identity 2 C44 (C11 + C12) = (C11 - C12)(C11 + 3 C12).  The energy of
homogeneous deformations of a periodic crystal, divided by the volume, must reproduce them.
Uniaxial [100] strain of a crystal changes every bond and every bond angle term by the same
amount, which gives the exact closed form used below.  The remaining pins are invariances, the
gradient against central differences and the zero of a relaxed structure.
"""
import numpy as np
import pytest

import synth
from oracle import vff


def pure(nx, ny, nz, periodic, alpha=300.0, beta=80.0, a=0.5431, a_box=None):
    vp = synth.VFFParams(np.array([a]), np.array([alpha]), np.array([beta]))
    spec = synth.lattice_spec(nx, ny, nz, periodic, seed=0, a_nm=a if a_box is None else a_box)
    return spec, vp, vff.geometry(spec, vp)


def curvature(g, V, F_of_eps, eps=1e-4):
    z = np.zeros_like(g.x0)
    return (vff.energy(g, z, F_of_eps(eps)) + vff.energy(g, z, F_of_eps(-eps))) / eps ** 2 / V


def test_ideal_crystal_is_a_stationary_zero():
    spec, vp, g = pure(2, 2, 2, (1, 1, 1))
    z = np.zeros_like(g.x0)
    assert abs(vff.energy(g, z)) < 1e-24
    assert np.abs(vff.gradient(g, z)).max() < 1e-14


def test_elastic_constants_are_keatings():
    alpha, beta, a = 310.0, 75.0, 0.5431
    spec, vp, g = pure(2, 2, 2, (1, 1, 1), alpha, beta, a)
    V = 8 * a ** 3
    I = np.eye(3)
    ex = np.diag([1.0, 0.0, 0.0])
    bi = np.diag([1.0, 1.0, 0.0])
    sh = np.zeros((3, 3))
    sh[0, 1] = sh[1, 0] = 0.5                    # engineering shear gamma_xy = eps
    c11 = curvature(g, V, lambda e: I + e * ex)
    c11_12 = curvature(g, V, lambda e: I + e * bi) / 2
    c44_0 = curvature(g, V, lambda e: I + e * sh)
    assert abs(c11 - (alpha + 3 * beta) / a) < 1e-6 * c11
    assert abs((c11_12 - c11) - (alpha - beta) / a) < 1e-6 * c11
    assert abs(c44_0 - (alpha + beta) / a) < 1e-6 * c11
    # relaxed shear: the sublattices move; the energy drops to Keating's C44
    gam = 1e-3
    u, E, fmax = vff.relax(g, I + gam * sh)
    assert fmax < 1e-9
    c44 = 2 * E / gam ** 2 / V
    assert abs(c44 - 4 * alpha * beta / (a * (alpha + beta))) < 1e-5 * c44
    c12 = c11_12 - c11
    assert abs(2 * c44 * (c11 + c12) - (c11 - c12) * (c11 + 3 * c12)) < 1e-4 * c11 ** 2


@pytest.mark.parametrize("eps", [-0.03, 0.01, 0.05])
def test_uniaxial_strain_of_a_cluster_has_the_closed_form(eps):
    """Every bond term and every angle term equals (a^2/16)^2 ((1+eps)^2 - 1)^2 times its
    prefactor 3 alpha/(8 d^2) or 3 beta/(8 d^2), with d^2 = 3a^2/16: E = a^2/128 (n_b alpha +
    n_angles beta) ((1+eps)^2 - 1)^2, exactly, for any block with free surfaces."""
    alpha, beta, a = 280.0, 70.0, 0.5431
    spec, vp, g = pure(3, 2, 4, (0, 1, 0), alpha, beta, a)
    n_b, n_ang = len(g.d), len(g.p)
    F = np.diag([1.0 + eps, 1.0, 1.0])
    E = vff.energy(g, np.zeros_like(g.x0), F)
    ref = a ** 2 / 128 * (n_b * alpha + n_ang * beta) * ((1 + eps) ** 2 - 1) ** 2
    assert abs(E - ref) < 1e-12 * ref


def test_gradient_matches_central_differences():
    spec = synth.lattice_spec(2, 2, 2, (1, 0, 1), seed=3, alloy_fraction=0.4)
    vp = synth.draw_vff_params(3)
    g = vff.geometry(spec, vp)
    u = synth.rng(4, 99).uniform(-0.01, 0.01, size=g.x0.shape)
    F = np.array([[1.01, 0.002, 0.0], [0.002, 0.995, 0.0], [0.0, 0.0, 1.0]])
    G = vff.gradient(g, u, F)
    h = 1e-6
    for idx in [(0, 0), (5, 1), (17, 2), (40, 0), (63, 1)]:
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        fd = (vff.energy(g, up, F) - vff.energy(g, um, F)) / (2 * h)
        assert abs(fd - G[idx]) < 1e-6 * max(1.0, abs(G[idx])), (idx, fd, G[idx])


def test_rigid_motions_cost_nothing():
    spec = synth.lattice_spec(2, 2, 2, (0, 0, 0), seed=5, alloy_fraction=0.5)
    vp = synth.draw_vff_params(5)
    g = vff.geometry(spec, vp)
    u = synth.rng(6, 99).uniform(-0.01, 0.01, size=g.x0.shape)
    E = vff.energy(g, u)
    assert abs(vff.energy(g, u + np.array([0.3, -0.1, 0.7])) - E) < 1e-12 * E
    th = 0.4
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    x = g.x0 + u
    assert abs(vff.energy(g, x @ R.T - g.x0) - E) < 1e-10 * E
    # forces of a free cluster sum to zero
    assert np.abs(vff.gradient(g, u).sum(axis=0)).max() < 1e-12 * np.abs(vff.gradient(g, u)).max()


def test_relaxed_alloy_bonds_and_slots():
    """A random Si/Ge alloy in a periodic box at the Si lattice constant: relaxation leaves no
    force, lowers the energy, and Ge-Ge bonds end longer than Si-Si bonds; the strain slots of
    the assembly's layout carry |r|/d - 1."""
    spec = synth.lattice_spec(2, 2, 2, (1, 1, 1), seed=7, alloy_fraction=0.5)
    vp = synth.draw_vff_params(7)
    g = vff.geometry(spec, vp)
    z = np.zeros_like(g.x0)
    E0 = vff.energy(g, z)
    u, E, fmax = vff.relax(g)
    assert fmax < 1e-9 and E < E0
    r = np.linalg.norm(vff.bond_vectors(g, u), axis=1)
    sa, sb = spec.species[g.bonds.a], spec.species[g.bonds.b]
    assert r[(sa == 1) & (sb == 1)].mean() > r[(sa == 0) & (sb == 0)].mean()
    st = vff.bond_strain(g, u)
    assert st.shape == (16 * spec.ncells,)
    np.testing.assert_allclose(st[g.bonds.slot], r / g.d - 1.0, rtol=0, atol=1e-15)


def test_bond_strain_of_a_scaled_pure_crystal():
    spec, vp, g = pure(2, 1, 3, (1, 1, 0), a_box=0.55)
    st = vff.bond_strain(g, np.zeros_like(g.x0))
    np.testing.assert_allclose(st[g.bonds.slot], 0.55 / 0.5431 - 1.0, rtol=0, atol=1e-14)
    missing = np.setdiff1d(np.arange(16 * spec.ncells), g.bonds.slot)
    assert len(missing) > 0 and np.all(st[missing] == 0)
