"""Pins for the oracle's lattice, CSR assembly and bulk folding.

* bond counts: periodic 16 n^3; hard wall 16n^3 - 12n^2 + 3n (derived below by counting the
  bonds that leave the block), checked by the k-d tree search;
* Hermiticity;
* periodic supercell spectrum = bulk two-atom H(k) spectra folded onto the supercell
  (translation symmetry; exact), with and without Bloch phases, with and without spin-orbit;
* bulk diamond Gamma-point closed forms (sp3s*): p states E_p +- (4/3)(V_pp_sigma + 2 V_pp_pi),
  three-fold each, and the two s/s* 2x2 blocks;
* spin-orbit: L.sigma on p has eigenvalues +1 (x4) and -2 (x2); every level of a spin-orbit
  H without a Bloch phase is two-fold (Kramers);
* a uniform bond strain eps equals scaling every two-centre integral by (1+eps)^-2.
"""
import numpy as np
import pytest

import synth
from oracle import lattice, hamiltonian, bulk, eigs
from oracle.hamiltonian import so_matrix


def hard_wall_bonds(n):
    # every A atom has 4 bonds in the infinite crystal; a bond is lost when its B end leaves
    # the block.  Along a direction the A->B step is +-a/4; a B end leaves through the low
    # face when the A atom sits at the low face (x = 0) and the step is negative, and the
    # same for the high face is impossible (A coordinates are 0 or 2 mod 4, B end <= 4n-1).
    # Counting by inclusion-exclusion over the three axes gives 16n^3 - 12n^2 + 3n.
    return 16 * n ** 3 - 12 * n ** 2 + 3 * n


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_bond_counts(n):
    assert len(lattice.find_bonds(n, n, n, (1, 1, 1)).a) == 16 * n ** 3
    assert len(lattice.find_bonds(n, n, n, (0, 0, 0)).a) == hard_wall_bonds(n)


def test_bond_count_brute_force_small():
    # O(N^2) distance check for n=2 hard wall, independent of the k-d tree
    pos = lattice.positions(2, 2, 2)
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    assert (d2 == 3).sum() // 2 == hard_wall_bonds(2)


def test_mixed_boundaries_and_each_slot_once():
    b = lattice.find_bonds(3, 2, 4, (1, 2, 0))
    assert len(np.unique(b.slot)) == len(b.slot)
    # x, y periodic: only z faces lose bonds -> per A atom at z = 0 two bonds with -z step
    ncells = 3 * 2 * 4
    assert len(b.a) == 16 * ncells - 2 * 2 * (3 * 2)


@pytest.mark.parametrize("basis,so,kv", [(5, False, None), (10, False, None), (10, True, None),
                                          (5, False, (0.31, -0.17, 0.05)), (10, True, (0.2, 0.1, -0.3))])
def test_hermitian(basis, so, kv):
    spec = synth.lattice_spec(2, 2, 2, (2, 2, 0) if kv else (0, 1, 0), seed=4, alloy_fraction=0.4,
                              strain_amp=0.02)
    p = synth.draw_tb_params(4, basis, 2)
    U = np.random.default_rng(0).uniform(-0.1, 0.1, spec.natoms)
    H = hamiltonian.assemble(spec, p, U_atom=U, kvec=kv, spin_orbit=so)
    assert abs(H - H.conj().T).max() < 1e-14


@pytest.mark.parametrize("basis,so,n", [(5, False, 2), (10, False, 2), (5, True, 2), (10, True, 1), (5, False, 3)])
def test_periodic_supercell_is_folded_bulk(basis, so, n):
    spec = synth.lattice_spec(n, n, n, (1, 1, 1), seed=7)
    p = synth.draw_tb_params(7, basis, 1)
    H = hamiltonian.assemble(spec, p, spin_orbit=so)
    ev = np.linalg.eigvalsh(H.toarray())
    ref = bulk.folded_spectrum(p, n, n, n, spec.a_nm, spin_orbit=so)
    np.testing.assert_allclose(ev, ref, atol=1e-11)


def test_bloch_supercell_is_folded_bulk_at_k0():
    spec = synth.lattice_spec(2, 2, 1, (2, 2, 2), seed=8)
    p = synth.draw_tb_params(8, 10, 1)
    k0 = np.array([0.37, -0.21, 0.44])
    H = hamiltonian.assemble(spec, p, kvec=k0)
    ev = np.linalg.eigvalsh(H.toarray())
    np.testing.assert_allclose(ev, bulk.folded_spectrum(p, 2, 2, 1, spec.a_nm, k0=k0), atol=1e-11)


def test_gamma_closed_forms_sp3s():
    p = synth.draw_tb_params(12, 5, 1)
    Es, Ep, _, Ess = p.onsite[0]
    V = p.V[0, 0]
    ss, sSsS, sS, pps, ppp = V[0], V[1], V[2], V[7], V[8]
    c = 4.0 / 3.0 * (pps + 2 * ppp)
    expect = [Ep + c] * 3 + [Ep - c] * 3
    expect += list(np.linalg.eigvalsh([[Es + 4 * ss, 4 * sS], [4 * sS, Ess + 4 * sSsS]]))
    expect += list(np.linalg.eigvalsh([[Es - 4 * ss, -4 * sS], [-4 * sS, Ess - 4 * sSsS]]))
    hk = bulk.bulk_hk(p, np.zeros(3), synth.SI_A_NM)
    np.testing.assert_allclose(np.linalg.eigvalsh(hk), np.sort(expect), atol=1e-12)
    # and these ten values appear in the periodic 2^3 supercell spectrum
    spec = synth.lattice_spec(2, 2, 2, (1, 1, 1), seed=12)
    ev = np.linalg.eigvalsh(hamiltonian.assemble(spec, p).toarray())
    for e in expect:
        assert np.min(np.abs(ev - e)) < 1e-11


def test_spin_orbit_p_block_and_bulk_gamma():
    M = so_matrix(10)
    w = np.linalg.eigvalsh(M)
    np.testing.assert_allclose(w[:2], [-2, -2], atol=1e-14)
    np.testing.assert_allclose(w[-4:], [1, 1, 1, 1], atol=1e-14)
    np.testing.assert_allclose(w[2:-4], 0, atol=1e-14)
    p = synth.draw_tb_params(13, 5, 1)
    lam = p.lambda_so[0]
    Ep = p.onsite[0, 1]
    c = 4.0 / 3.0 * (p.V[0, 0, 7] + 2 * p.V[0, 0, 8])
    ev = np.linalg.eigvalsh(bulk.bulk_hk(p, np.zeros(3), synth.SI_A_NM, spin_orbit=True))
    for sgn in (+1, -1):
        for shift, mult in ((lam, 4), (-2 * lam, 2)):
            assert np.sum(np.abs(ev - (Ep + sgn * c + shift)) < 1e-11) == mult


def test_kramers_degeneracy():
    spec = synth.lattice_spec(2, 1, 2, (0, 1, 0), seed=5, alloy_fraction=0.5, strain_amp=0.02)
    p = synth.draw_tb_params(5, 10, 2)
    ev = np.linalg.eigvalsh(hamiltonian.assemble(spec, p, spin_orbit=True).toarray())
    np.testing.assert_allclose(ev[0::2], ev[1::2], atol=1e-11)


def test_uniform_strain_is_integral_scaling():
    spec = synth.lattice_spec(2, 2, 2, (0, 1, 1), seed=9, alloy_fraction=0.3)
    p = synth.draw_tb_params(9, 10, 2)
    eps = 0.015
    spec.strain[:] = eps
    H1 = hamiltonian.assemble(spec, p)
    spec.strain[:] = 0.0
    p2 = synth.TBParams(p.basis, p.onsite, p.V * (1 + eps) ** -2, p.lambda_so)
    H2 = hamiltonian.assemble(spec, p2)
    assert abs(H1 - H2).max() < 1e-14


def test_potential_shifts_diagonal_only():
    spec = synth.lattice_spec(2, 2, 2, (1, 1, 0), seed=10)
    p = synth.draw_tb_params(10, 5, 1)
    U = np.linspace(-0.3, 0.2, spec.natoms)
    D = hamiltonian.assemble(spec, p, U_atom=U) - hamiltonian.assemble(spec, p)
    np.testing.assert_allclose(D.diagonal(), np.tile(U, 5), atol=1e-15)
    assert abs(D - np.diag(D.diagonal())).max() < 1e-15


def test_hx_rows_sample_matches_full_product():
    spec = synth.lattice_spec(3, 2, 2, (0, 2, 1), seed=3, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(3, 10, 2)
    kv = (0.0, 0.4, 0.0)
    H = hamiltonian.assemble(spec, p, kvec=kv, spin_orbit=True)
    x = synth.random_vectors(1, H.shape[0], dtype=complex)[0]
    atoms = np.array([0, 5, 17, spec.natoms - 1])
    rows, vals = hamiltonian.hx_rows(spec, p, x, atoms, kvec=kv, spin_orbit=True)
    np.testing.assert_allclose(vals, (H @ x)[rows], atol=1e-13)
