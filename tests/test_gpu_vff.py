"""Valence-force-field strain relaxation on the device against the Keating oracle.

* energy and forces at random displacements and a sheared box, element by element against
  the oracle's energy and -gradient (FP64: 1e-12 of the largest force, 1e-12 relative energy),
  on alloys with hard-wall, periodic and one-cell periodic axes (ragged tails: cell counts that
  are not multiples of the CTA width);
* the closed forms the oracle is pinned to, now on the device: the ideal crystal has zero energy
  and force, and uniaxial strain of a free block has Keating's exact energy;
* relaxation: the relaxed energy equals the oracle's (both to forces below 1e-10 eV/nm; the
  minimum is unique up to rigid motions, so energies and bond strains are compared), the relaxed
  bond strains agree to 1e-9 per slot, and no force is left above the tolerance;
* the relaxed strains feed the tight-binding assembly: H·X with them equals the oracle's H built
  from the oracle's own relaxed strains.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import hamiltonian, vff  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1003_4570_gb300 import omen
    return omen.omen_create(0, torch.cuda.current_stream().cuda_stream)


SHEAR = np.array([[1.01, 0.002, 0.0], [0.002, 0.995, 0.0], [0.0, 0.0, 1.0]])


def soa(u):
    """(natoms, 3) -> device [3][natoms]."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(u, float).T)).cuda()


def aos(t):
    return t.cpu().numpy().reshape(3, -1).T


@pytest.mark.parametrize("dims,periodic", [((4, 3, 5), (1, 0, 1)), ((5, 4, 7), (0, 0, 0)), ((3, 3, 3), (1, 1, 1)),
                                           ((1, 2, 3), (1, 1, 0))])
def test_energy_and_forces_match_oracle(ctx, dims, periodic):
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(*dims, periodic, seed=3, alloy_fraction=0.4)
    vp = synth.draw_vff_params(3)
    g = vff.geometry(spec, vp)
    u = synth.rng(4, 99).uniform(-0.01, 0.01, size=g.x0.shape)
    lat = omen.omen_build_lattice(ctx, spec)
    ud = soa(u)
    f = torch.empty_like(ud)
    E = omen.omen_vff_energy_forces(ctx, lat, vp, ud, F=SHEAR, force_dev=f)
    E_ref = vff.energy(g, u, SHEAR)
    G_ref = vff.gradient(g, u, SHEAR)
    assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
    np.testing.assert_allclose(aos(f), -G_ref, atol=1e-12 * np.abs(G_ref).max(), rtol=0)
    # no deformation given = identity
    E_id = omen.omen_vff_energy_forces(ctx, lat, vp, ud)
    assert abs(E_id - vff.energy(g, u)) <= 1e-12 * abs(E_id)


def test_keating_closed_forms_on_device(ctx):
    from paper_1003_4570_gb300 import omen
    alpha, beta, a = 280.0, 70.0, 0.5431
    vp = synth.VFFParams(np.array([a]), np.array([alpha]), np.array([beta]))
    # ideal periodic crystal: a stationary zero
    spec = synth.lattice_spec(3, 2, 4, (1, 1, 1), seed=0, a_nm=a)
    lat = omen.omen_build_lattice(ctx, spec)
    z = torch.zeros((3, spec.natoms), dtype=torch.float64, device="cuda")
    f = torch.empty_like(z)
    E = omen.omen_vff_energy_forces(ctx, lat, vp, z, force_dev=f)
    assert abs(E) < 1e-24 and f.abs().max().item() < 1e-14
    # uniaxial [100] strain of a block with free surfaces: every bond and angle term is
    # (a^2/16)^2 ((1+eps)^2 - 1)^2 times its prefactor, E = a^2/128 (n_b alpha + n_ang beta) (...)^2
    spec = synth.lattice_spec(3, 2, 4, (0, 1, 0), seed=0, a_nm=a)
    lat = omen.omen_build_lattice(ctx, spec)
    g = vff.geometry(spec, vp)
    z = torch.zeros((3, spec.natoms), dtype=torch.float64, device="cuda")
    for eps in (-0.03, 0.05):
        E = omen.omen_vff_energy_forces(ctx, lat, vp, z, F=np.diag([1.0 + eps, 1.0, 1.0]))
        ref = a ** 2 / 128 * (len(g.d) * alpha + len(g.p) * beta) * ((1 + eps) ** 2 - 1) ** 2
        assert abs(E - ref) < 1e-12 * ref


@pytest.mark.parametrize("dims,periodic,F", [((4, 3, 5), (1, 0, 1), SHEAR), ((12, 12, 12), (1, 1, 0), None)])
def test_relaxation_matches_oracle(ctx, dims, periodic, F):
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(*dims, periodic, seed=11, alloy_fraction=0.3)
    vp = synth.draw_vff_params(11)
    g = vff.geometry(spec, vp)
    u_ref, E_ref, fmax_ref = vff.relax(g, F, gtol=1e-10)
    assert fmax_ref < 1e-10
    lat = omen.omen_build_lattice(ctx, spec)
    ud = torch.zeros((3, spec.natoms), dtype=torch.float64, device="cuda")
    st = torch.empty(16 * spec.ncells, dtype=torch.float64, device="cuda")
    info, _ = omen.omen_relax_vff(ctx, lat, vp, ud, F=F, gtol=1e-10, max_iter=20000, strain_dev=st)
    assert info["converged"] == 1 and info["max_force"] < 1e-10, info
    assert info["energy"] < info["energy_start"]
    assert abs(info["energy"] - E_ref) <= 1e-10 * E_ref
    # the device's own forces at its relaxed displacements, and the oracle's there
    u = aos(ud)
    assert np.abs(vff.gradient(g, u, F)).max() < 1e-9
    s_ref = vff.bond_strain(g, u_ref, F)
    np.testing.assert_allclose(st.cpu().numpy(), s_ref, atol=1e-9, rtol=0)
    # a second call from the relaxed state stops at once
    info2, _ = omen.omen_relax_vff(ctx, lat, vp, ud, F=F, gtol=1e-10, max_iter=20000)
    assert info2["iterations"] == 0 and info2["converged"] == 1


def test_relaxed_strain_feeds_assembly(ctx):
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(3, 4, 5, (1, 1, 0), seed=21, alloy_fraction=0.5)
    vp = synth.draw_vff_params(21)
    p = synth.draw_tb_params(21, 10, 2)
    g = vff.geometry(spec, vp)
    u_ref, _, _ = vff.relax(g, gtol=1e-10)
    spec.strain = vff.bond_strain(g, u_ref)
    H = hamiltonian.assemble(spec, p)
    lat = omen.omen_build_lattice(ctx, synth.lattice_spec(3, 4, 5, (1, 1, 0), seed=21, alloy_fraction=0.5))
    ud = torch.zeros((3, spec.natoms), dtype=torch.float64, device="cuda")
    st = torch.empty(16 * spec.ncells, dtype=torch.float64, device="cuda")
    omen.omen_relax_vff(ctx, lat, vp, ud, gtol=1e-10, strain_dev=st)
    omen.omen_lattice_set_strain(ctx, lat, st)
    for mf in (False, True):
        ham = omen.omen_assemble_H(ctx, lat, p, matrix_free=mf)
        x = synth.random_vectors(5, H.shape[0])[0]
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        omen.omen_hx(ctx, ham, xd, yd)
        ref = H @ x
        # strains agree to ~1e-12, the Harrison factor turns that into ~1e-12 relative
        np.testing.assert_allclose(yd.cpu().numpy(), ref, atol=1e-10 * np.abs(ref).max(), rtol=0)
