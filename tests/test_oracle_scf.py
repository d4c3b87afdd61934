"""Pins for the delta-layer workload and the oracle's self-consistent loop.

* the stored gapped parameter draw is what the golden script accepts, and its bulk bands do
  have the stored gap (re-checked on a coarse folded grid);
* the donor sheet on the grid carries exactly e N_s per unit area;
* the oracle SCF reaches its fixed point (max |phi_out - phi| < tol) and conserves charge:
  electrons per atom sum to the electron count, and the total charge is neutral;
* the physics of the coupling between the Poisson potential and the Hamiltonian (Section
  III-A items 2-3), checked on the converged potential so that a flipped sign of the
  electron's potential energy (U = -phi) or of the electron charge fails:
  - discrete Gauss law: for the 7-point operator with phi = 0 on both z ends, the interior
    charge equals eps0 eps_r hx hy / hz times the sum of phi over the first and last interior
    planes.  A neutral fixed point has (almost) no net charge, so the end fields cancel; with
    the electron charge's sign flipped the net charge would be twice the donors';
  - electrons (charge -e) are drawn to high potential: the atomic plane holding the most
    electrons sits at the donor sheet, and the electron-weighted mean of phi at the atoms
    exceeds the plain mean; with U = +phi they would be pushed away from the sheet;
  - the positive donor sheet makes phi a hill with its top at the sheet.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import bulk, charge, poisson, scf

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gapped_si_params.json")


def test_gapped_params_match_golden():
    g = json.load(open(GOLD))
    assert g["seed"] == synth.GAPPED_SI_SEED
    assert abs(g["E_v"] - synth.GAPPED_SI_EV) < 1e-12 and abs(g["E_c"] - synth.GAPPED_SI_EC) < 1e-12
    p = synth.gapped_si_params()
    ks = bulk.folded_wavevectors(3, 3, 3, synth.SI_A_NM)
    ev = np.array([np.linalg.eigvalsh(bulk.bulk_hk(p, k, synth.SI_A_NM)) for k in ks])
    # a coarser grid samples a subset of k: edges can only be at or inside the fine-grid edges
    assert ev[:, 3].max() <= g["E_v"] + 1e-9 and ev[:, 4].min() >= g["E_c"] - 1e-9
    assert g["gap"] >= 0.5


def test_donor_sheet_normalisation():
    rho = synth.donor_rho_on_grid(7.3e13, 1.2, 4, 3, 60, 12.0)
    hz = 12.0 / 60 * 1e-9
    assert abs(rho[:, 0, 0].sum() * hz - synth.Q_E * 7.3e13 * 1e4) < 1e-12 * synth.Q_E * 7.3e17
    assert np.allclose(rho, rho[:, :1, :1])


def small_delta_case(nxy=1, nzc=12, ns=1e14):
    spec, p, (_, w) = synth.delta_layer(nxy, nzc, seed=5)
    a = spec.a_nm
    n = max(2, round(nxy * a / 0.2))
    grid = poisson.Grid(n, n, round(nzc * a / 0.2), nxy * a, nxy * a, nzc * a)
    rho_d = synth.donor_rho_on_grid(ns, w, grid.nx, grid.ny, grid.nz, grid.Lz_nm)
    ne = ns * (nxy * a * 1e-7) ** 2
    eg = synth.GAPPED_SI_EC - synth.GAPPED_SI_EV
    return dict(spec=spec, params=p, grid=grid, donor_rho=rho_d, n_electrons=ne, kT=8.617333262e-5 * 4,
                kpts=[(0.0, 0.0, 0.0)], kweights=[1.0], nev=8, sigma=synth.GAPPED_SI_EC - 0.4 * eg,
                e_cut=0.5 * (synth.GAPPED_SI_EC + synth.GAPPED_SI_EV))


def test_oracle_scf_fixed_point_and_neutrality():
    c = small_delta_case()
    phi, info = scf.scf(c["spec"], c["params"], c["grid"], c["donor_rho"], c["n_electrons"], c["kT"], c["kpts"],
                        c["kweights"], c["nev"], c["sigma"], c["e_cut"], mix=0.3, tol_V=1e-6, max_iter=200)
    assert info["dV_inf"] < 1e-6
    assert abs(info["n_atom"].sum() - c["n_electrons"]) < 1e-9
    hz = c["grid"].Lz_nm / c["grid"].nz * 1e-9
    area = c["grid"].Lx_nm * c["grid"].Ly_nm * 1e-18
    donors = c["donor_rho"][:, 0, 0].sum() * hz * area
    assert abs(donors - synth.Q_E * c["n_electrons"]) < 1e-9 * donors


@pytest.fixture(scope="module")
def converged_delta():
    c = small_delta_case()
    phi, info = scf.scf(c["spec"], c["params"], c["grid"], c["donor_rho"], c["n_electrons"], c["kT"], c["kpts"],
                        c["kweights"], c["nev"], c["sigma"], c["e_cut"], mix=0.3, tol_V=1e-8, max_iter=300,
                        mix_history=5)
    assert info["dV_inf"] < 1e-8
    return c, phi, info


def net_charge_from_end_fields(grid, phi):
    """Discrete Gauss law: summing the 7-point operator over all interior unknowns leaves only
    the z-boundary terms (the x, y differences telescope to zero on the periodic axes and
    phi = 0 on the z = 0, Lz planes), so sum_k rho_k V_cell = eps hx hy / hz * sum(phi_1 + phi_nz-1)."""
    hx, hy, hz = grid.h_m
    return poisson.EPS0 * grid.eps_r * hx * hy / hz * (phi[0].sum() + phi[-1].sum())


def check_coupling_physics(c, phi, info):
    grid = c["grid"]
    hx, hy, hz = grid.h_m
    q_donor = c["donor_rho"].sum() * hx * hy * hz
    # neutral: what is left is the few electrons on atoms within a spacing of the grounded planes
    assert abs(net_charge_from_end_fields(grid, phi)) < 1e-3 * q_donor
    pos = scf.atom_positions_nm(c["spec"])
    n = info["n_atom"]
    planes = np.unique(np.round(pos[:, 2], 9))
    per_plane = np.array([n[np.abs(pos[:, 2] - z) < 1e-6].sum() for z in planes])
    z_sheet = 0.5 * grid.Lz_nm
    _, w = synth.delta_layer(1, 12, seed=5)[2]
    assert abs(planes[per_plane.argmax()] - z_sheet) <= 0.25 * w
    phi_at = charge.gather(grid, phi, pos)
    assert (n * phi_at).sum() / n.sum() > phi_at.mean() + 0.1 * np.ptp(phi_at)
    prof = phi.reshape(grid.nz - 1, -1).mean(axis=1)
    z = np.arange(1, grid.nz) * grid.Lz_nm / grid.nz
    assert prof.max() > 0 and abs(z[prof.argmax()] - z_sheet) <= 0.25 * w
    assert prof.max() > 10 * np.abs(prof[[0, -1]]).max()


def test_oracle_scf_coupling_signs(converged_delta):
    check_coupling_physics(*converged_delta)


def test_oracle_scf_anderson_reaches_same_fixed_point():
    c = small_delta_case()
    args = (c["spec"], c["params"], c["grid"], c["donor_rho"], c["n_electrons"], c["kT"], c["kpts"], c["kweights"],
            c["nev"], c["sigma"], c["e_cut"])
    phi_lin, _ = scf.scf(*args, mix=0.3, tol_V=1e-8, max_iter=300)
    phi_and, info = scf.scf(*args, mix=0.3, tol_V=1e-8, max_iter=300, mix_history=5)
    assert info["dV_inf"] < 1e-8
    assert np.abs(phi_lin - phi_and).max() < 1e-7
