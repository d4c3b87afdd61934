"""Pins for the delta-layer workload and the oracle's self-consistent loop.

* the stored gapped parameter draw is what the golden script accepts, and its bulk bands do
  have the stored gap (re-checked on a coarse folded grid);
* the donor sheet on the grid carries exactly e N_s per unit area;
* the oracle SCF reaches its fixed point (max |phi_out - phi| < tol) and conserves charge:
  electrons per atom sum to the electron count, and the total charge is neutral.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import bulk, poisson, scf

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


def test_oracle_scf_anderson_reaches_same_fixed_point():
    c = small_delta_case()
    args = (c["spec"], c["params"], c["grid"], c["donor_rho"], c["n_electrons"], c["kT"], c["kpts"], c["kweights"],
            c["nev"], c["sigma"], c["e_cut"])
    phi_lin, _ = scf.scf(*args, mix=0.3, tol_V=1e-8, max_iter=300)
    phi_and, info = scf.scf(*args, mix=0.3, tol_V=1e-8, max_iter=300, mix_history=5)
    assert info["dV_inf"] < 1e-8
    assert np.abs(phi_lin - phi_and).max() < 1e-7
