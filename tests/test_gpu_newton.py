"""Newton–Raphson nonlinear Poisson on the GPU against the oracle (Section III-A item 3).

* state weights W_ni of eigenvector-like columns (real and Bloch-complex) against the
  oracle's, to rounding;
* the root of the nonlinear Poisson equation for the same frozen states, E_F, kT, phi_in and
  donor density, on grids with ragged sizes and periodic one-point axes: within 1e-9 V of the
  oracle's Newton root (both step to 1e-12 V);
* no states: the root is the linear Poisson solution (omen_poisson);
* the self-consistent loop with the Newton–Raphson Poisson step (Anderson mixing) against the
  oracle loop with the same reading, on the 1x1x12-cell delta layer at 77 K: converged
  potentials within 1e-6 V, Fermi levels within 1e-6 eV, and the same fixed point as the loop
  with the linear Poisson step.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import newton, poisson, scf  # noqa: E402
from test_oracle_scf import small_delta_case  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1003_4570_gb300 import omen
    return omen.omen_create(0, torch.cuda.current_stream().cuda_stream)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_state_weights_match_oracle(ctx):
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(2, 3, 4, (2, 2, 0), seed=9)
    lat = omen.omen_build_lattice(ctx, spec)
    p = synth.draw_tb_params(9, 10, 1)
    rng = np.random.default_rng(4)
    for k in (None, (0.3, 0.1, 0.0)):
        ham = omen.omen_assemble_H(ctx, lat, p, k=k)
        psi = rng.normal(size=(5, ham.nrows))
        if ham.is_complex:
            psi = psi + 1j * rng.normal(size=(5, ham.nrows))
        wts = np.array([2.0, 0.5, 0.0, 1.0, 0.25])
        W = torch.empty((5, spec.natoms), dtype=torch.float64, device="cuda")
        omen.omen_state_weights(ctx, ham, dev(psi), 5, wts, W)
        ref = np.stack([newton.state_weights(psi[n][:, None], wts[n], spec.natoms)[:, 0] for n in range(5)])
        np.testing.assert_allclose(W.cpu().numpy(), ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("dims,grid_n", [((1, 1, 3), (3, 2, 12)), ((2, 3, 5), (5, 7, 27)), ((1, 2, 4), (1, 4, 17))])
def test_newton_root_matches_oracle(ctx, dims, grid_n):
    from paper_1003_4570_gb300 import omen
    g = np.random.default_rng(sum(dims))
    spec = synth.lattice_spec(*dims, (1, 1, 0), seed=3)
    a = spec.a_nm
    grid = poisson.Grid(*grid_n, dims[0] * a, dims[1] * a, dims[2] * a)
    pos = scf.atom_positions_nm(spec)
    nst = 9
    W = g.uniform(0, 0.05, size=(spec.natoms, nst))
    E = np.sort(g.uniform(-0.05, 0.05, nst))
    EF, kT = 0.004, 0.01
    phi_in = g.normal(scale=0.02, size=grid.shape)
    donor = np.abs(g.normal(scale=2e6, size=grid.shape))
    prob = newton.Problem(grid, pos, W, E, EF, kT, phi_in, donor)
    ref, steps = newton.solve(prob, phi_in, tol=1e-12)
    lat = omen.omen_build_lattice(ctx, spec)
    phi = dev(phi_in.copy())
    info, st = omen.omen_poisson_newton(ctx, lat, grid, E, dev(W.T), EF, kT, dev(phi_in), dev(donor), phi, tol_V=1e-12)
    assert info["converged"] == 1 and info["iterations"] <= len(steps) + 2, (info, steps)
    np.testing.assert_allclose(phi.cpu().numpy(), ref, atol=1e-9, rtol=0)


def test_newton_without_states_is_the_linear_solve(ctx):
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(1, 1, 6, (1, 1, 0), seed=1)
    a = spec.a_nm
    grid = poisson.Grid(4, 4, 30, a, a, 6 * a)
    rho = np.abs(np.random.default_rng(2).normal(size=grid.shape)) * 1e6
    lat = omen.omen_build_lattice(ctx, spec)
    z = dev(np.zeros(grid.shape))
    phi = dev(np.zeros(grid.shape))
    W = torch.zeros((1, spec.natoms), dtype=torch.float64, device="cuda")
    info, _ = omen.omen_poisson_newton(ctx, lat, grid, [0.0], W, 0.0, 0.01, z, dev(rho), phi, tol_V=1e-12)
    assert info["converged"] == 1 and info["iterations"] <= 2
    ref = poisson.solve_direct(grid, rho)
    np.testing.assert_allclose(phi.cpu().numpy(), ref, atol=1e-10 * np.abs(ref).max(), rtol=0)


def test_scf_with_newton_poisson_matches_oracle(ctx):
    from paper_1003_4570_gb300 import omen
    c = small_delta_case()
    kT = 8.617333262e-5 * 77.0
    args = (c["spec"], c["params"], c["grid"], c["donor_rho"], c["n_electrons"], kT, c["kpts"], c["kweights"], 16,
            c["sigma"], c["e_cut"])
    phi_ref, info_ref = scf.scf(*args, mix=1.0, tol_V=1e-8, max_iter=120, mix_history=5, poisson_mode="newton")
    phi_lin, _ = scf.scf(*args, mix=0.3, tol_V=1e-9, max_iter=200, mix_history=5)
    assert np.abs(phi_ref - phi_lin).max() < 1e-6          # one fixed point for both Poisson steps
    lat = omen.omen_build_lattice(ctx, c["spec"])
    phi = torch.zeros(c["grid"].shape, dtype=torch.float64, device="cuda")
    info, st = omen.omen_scf(ctx, lat, c["params"], c["grid"], phi, dev(c["donor_rho"]), c["n_electrons"], kT,
                             c["kpts"], c["kweights"], 16, c["sigma"], c["e_cut"], eig_tol=1e-10, eig_block=4,
                             eig_basis=64, mix=1.0, tol_V=1e-8, max_iter=120, mix_history=5, poisson_newton=True)
    assert info["converged"] == 1, info
    assert abs(info["iterations"] - info_ref["iterations"]) <= 5, (info["iterations"], info_ref["iterations"])
    np.testing.assert_allclose(phi.cpu().numpy(), phi_ref, atol=1e-6, rtol=0)
    assert abs(info["E_F"] - info_ref["E_F"]) < 1e-6
