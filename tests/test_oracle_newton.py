"""Pins of the Newton–Raphson nonlinear Poisson oracle (Section III-A item 3).

* the Jacobian equals central differences of the residual (a dropped term, a transposed
  gather/deposit pair or a wrong sign of the level shift fails it);
* electrons are drawn to higher potential: raising phi everywhere raises the predicted count;
* with no states the nonlinear equation is the linear one, and for a uniform sheet of charge
  on one grid plane its root is the exact piecewise-linear discrete solution;
* a brute-force root of F on a small grid (scipy's hybrid Powell method, no Jacobian) is the
  Newton root, and the last Newton steps shrink quadratically;
* consistency: at the potential the states were computed in, the predicted density is the
  states' density, so at a self-consistent potential (from the oracle's linear-Poisson loop) the
  Newton root is that potential.
"""
import numpy as np
import pytest
import scipy.optimize as so

import synth
from oracle import charge, newton, poisson, scf
from test_oracle_scf import small_delta_case


def random_problem(seed=3, nstates=7, grid=None, nzc=3):
    g = np.random.default_rng(seed)
    spec = synth.lattice_spec(1, 1, nzc, (1, 1, 0), seed=seed)
    a = spec.a_nm
    grid = grid or poisson.Grid(3, 2, 4 * nzc, a, a, nzc * a)
    pos = scf.atom_positions_nm(spec)
    W = g.uniform(0, 0.05, size=(spec.natoms, nstates))
    E = np.sort(g.uniform(-0.05, 0.05, nstates))
    phi_in = g.normal(scale=0.02, size=grid.shape)
    donor = np.abs(g.normal(scale=2e6, size=grid.shape))
    return newton.Problem(grid, pos, W, E, 0.0, 0.01, phi_in, donor), phi_in


def test_jacobian_matches_central_differences():
    prob, phi_in = random_problem()
    phi = phi_in + np.random.default_rng(9).normal(scale=0.01, size=phi_in.shape)
    J = prob.jacobian(phi).toarray()
    h = 1e-6
    for j in (0, 5, 17, 30):
        e = np.zeros(phi.size)
        e[j] = h
        col = (prob.residual(phi.ravel() + e) - prob.residual(phi.ravel() - e)) / (2 * h)
        np.testing.assert_allclose(J[:, j], col, rtol=1e-6, atol=1e-6 * np.abs(J).max())


def test_electrons_follow_the_potential():
    prob, phi_in = random_problem()
    n0, s0 = prob.density(phi_in)
    n1, _ = prob.density(phi_in + 0.01)
    assert np.all(n1 >= n0) and n1.sum() > n0.sum() and np.all(s0 >= 0)


def test_no_states_gives_the_exact_sheet_potential():
    """A uniform sheet sigma_s on grid plane k0 with phi = 0 at both ends: phi(z) = sigma_s/eps *
    z (L - z0) / L below the sheet and sigma_s/eps * z0 (L - z) / L above it, exact for the
    3-point difference (piecewise linear)."""
    grid = poisson.Grid(2, 3, 12, 1.0, 1.0, 6.0)
    spec = synth.lattice_spec(1, 1, 2, (1, 1, 0), seed=0)
    pos = scf.atom_positions_nm(spec)
    k0 = 5
    sig = 3e-3                                    # C/m^2
    hz = grid.h_m[2]
    donor = np.zeros(grid.shape)
    donor[k0 - 1] = sig / hz
    prob = newton.Problem(grid, pos, np.zeros((spec.natoms, 2)), np.zeros(2), 0.0, 0.01, np.zeros(grid.shape), donor)
    phi, steps = newton.solve(prob, np.zeros(grid.shape))
    L = grid.Lz_nm * 1e-9
    z = np.arange(1, grid.nz) * hz
    z0 = k0 * hz
    eps = poisson.EPS0 * grid.eps_r
    exact = np.where(z <= z0, sig / eps * z * (L - z0) / L, sig / eps * z0 * (L - z) / L)
    np.testing.assert_allclose(phi[:, 0, 0], exact, rtol=1e-12, atol=1e-14)
    assert len(steps) <= 2                        # linear: one step, then a zero step


def test_newton_root_is_the_brute_force_root():
    prob, phi_in = random_problem(seed=5, nzc=2)
    phi, steps = newton.solve(prob, phi_in, tol=1e-13)
    scale = 1.0 / np.abs(prob.residual(phi_in)).max()
    sol = so.root(lambda v: scale * prob.residual(v), phi_in.ravel(), method="hybr", tol=1e-14)
    assert np.abs(scale * prob.residual(sol.x)).max() < 1e-12      # a root, found without J
    np.testing.assert_allclose(phi.ravel(), sol.x, atol=1e-11, rtol=0)
    # quadratic convergence near the root
    big = [s for s in steps if s > 1e-12]
    if len(big) >= 3:
        assert big[-1] <= 10 * big[-2] ** 2 / big[-3] + 1e-12


def test_self_consistent_potential_is_a_newton_root():
    c = small_delta_case()
    phi_sc, info = scf.scf(c["spec"], c["params"], c["grid"], c["donor_rho"], c["n_electrons"], c["kT"], c["kpts"],
                           c["kweights"], c["nev"], c["sigma"], c["e_cut"], mix=0.3, tol_V=1e-10, max_iter=300,
                           mix_history=5)
    # the states of the converged potential, frozen
    from oracle import hamiltonian, lattice
    spec = c["spec"]
    pos = scf.atom_positions_nm(spec)
    bonds = lattice.find_bonds(spec.nx, spec.ny, spec.nz, spec.periodic)
    H = hamiltonian.assemble(spec, c["params"], U_atom=-charge.gather(c["grid"], phi_sc, pos), kvec=c["kpts"][0],
                             bonds=bonds)
    w, V = scf.nearest_states(H, c["sigma"], c["nev"])
    m = w > c["e_cut"]
    W = newton.state_weights(V[:, m], 2.0, spec.natoms)
    prob = newton.Problem(c["grid"], pos, W, w[m], info["E_F"], c["kT"], phi_sc, c["donor_rho"])
    n, _ = prob.density(phi_sc)
    np.testing.assert_allclose(n, info["n_atom"], rtol=0, atol=1e-12)
    phi, _ = newton.solve(prob, phi_sc)
    assert np.abs(phi - phi_sc).max() < 1e-8
