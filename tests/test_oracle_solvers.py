"""Pins for the oracle's eigensolvers, Poisson solver and charge routines.

* plain Lanczos (lowest) and folded-spectrum Lanczos (nearest sigma) against a dense
  Hermitian eigensolve and ARPACK shift-invert, on a small random alloy;
* Poisson: a uniform charge sheet between grounded z ends gives a piecewise-linear phi, for
  which the 7-point stencil is exact; a discrete Laplacian eigenmode sin(pi k z/L) cos(2 pi m x/Lx)
  with its exact discrete eigenvalue; CG equals the direct solve;
* charge: sum rule, monotone N(E_F), bisection hits the target, deposit conserves charge and
  gather is its adjoint.
"""
import numpy as np
import pytest

import synth
from oracle import hamiltonian, eigs, poisson, charge


@pytest.fixture(scope="module")
def small_alloy():
    spec = synth.lattice_spec(2, 2, 2, (0, 0, 0), seed=21, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(21, 10, 2)
    H = hamiltonian.assemble(spec, p)
    w, V = eigs.dense_eigh(H)
    return H, w, V


def test_lanczos_lowest(small_alloy):
    H, w, _ = small_alloy
    v0 = synth.start_block(1, H.shape[0])[0]
    lam, X, m = eigs.lowest(H, 6, v0, maxiter=H.shape[0], tol=1e-11)
    np.testing.assert_allclose(lam, w[:6], atol=1e-9)
    assert np.all(eigs.residual_norms(H, lam, X) < 1e-8)


def test_folded_nearest_sigma(small_alloy):
    H, w, _ = small_alloy
    sigma = 0.5 * (w[0] + w[-1]) + 0.37
    ref = eigs.nearest(w, sigma, 8)
    v0 = synth.start_block(2, H.shape[0])[0]
    lam, X, m = eigs.folded(H, sigma, 8, v0, maxiter=H.shape[0], tol=1e-13)
    np.testing.assert_allclose(lam, ref, atol=1e-9)
    si, _ = eigs.nearest_shift_invert(H, sigma, 8)
    np.testing.assert_allclose(si, ref, atol=1e-9)


def test_nearest_tie_rule():
    assert list(eigs.nearest([-1.0, 1.0, 3.0], 0.0, 1)) == [-1.0]
    assert list(eigs.nearest([0.5, -0.2, 2.0, 0.1], 0.0, 3)) == [-0.2, 0.1, 0.5]


@pytest.fixture
def grid():
    return poisson.Grid(5, 4, 30, 2.0, 1.6, 12.0, eps_r=11.7)


def test_poisson_sheet_exact(grid):
    sigma_s = 3.0e-3                       # C/m^2
    k0 = 11
    hz = grid.h_m[2]
    rho = np.zeros(grid.shape)
    rho[k0 - 1] = sigma_s / hz
    phi = poisson.solve_direct(grid, rho)
    L = grid.Lz_nm * 1e-9
    z = np.arange(1, grid.nz) * hz
    z0 = k0 * hz
    exact = np.where(z <= z0, z * (L - z0) / L, z0 * (L - z) / L) * sigma_s / (poisson.EPS0 * grid.eps_r)
    np.testing.assert_allclose(phi, np.broadcast_to(exact[:, None, None], grid.shape), rtol=1e-10, atol=1e-14)


def test_poisson_discrete_mode_and_cg(grid):
    hx, hy, hz = grid.h_m
    kz, mx = 3, 2
    z = np.arange(1, grid.nz) * hz
    x = np.arange(grid.nx) * hx
    L, Lx = grid.Lz_nm * 1e-9, grid.Lx_nm * 1e-9
    mode = np.sin(np.pi * kz * z / L)[:, None, None] * np.cos(2 * np.pi * mx * x / Lx)[None, None, :]
    mode = np.broadcast_to(mode, grid.shape)
    lam = (2 - 2 * np.cos(np.pi * kz / grid.nz)) / hz ** 2 + (2 - 2 * np.cos(2 * np.pi * mx / grid.nx)) / hx ** 2
    rho = lam * mode * poisson.EPS0 * grid.eps_r
    np.testing.assert_allclose(poisson.solve_direct(grid, rho), mode, atol=1e-12)
    phi_cg, it = poisson.solve_cg(grid, rho, rtol=1e-13)
    np.testing.assert_allclose(phi_cg, mode, atol=1e-11)
    assert it > 0


def test_charge_sum_rule_and_fermi():
    g = np.random.default_rng(5)
    natoms, nb, ns = 7, 3, 4
    psi = g.normal(size=(nb * natoms, ns)) + 1j * g.normal(size=(nb * natoms, ns))
    psi /= np.linalg.norm(psi, axis=0)
    occ = g.uniform(0, 2, ns)
    n = charge.atom_density(psi, occ, natoms)
    assert abs(n.sum() - occ.sum()) < 1e-12
    evals = [np.sort(g.uniform(-1, 1, 20)) for _ in range(3)]
    w = [0.5, 0.25, 0.25]
    kT = 0.01
    counts = [charge.electron_count(evals, w, e, kT, 2) for e in np.linspace(-1.2, 1.2, 50)]
    assert np.all(np.diff(counts) >= 0)
    EF = charge.fermi_level(evals, w, 7.3, kT, 2)
    assert abs(charge.electron_count(evals, w, EF, kT, 2) - 7.3) < 1e-9


def test_deposit_conserves_and_gather_is_adjoint(grid):
    g = np.random.default_rng(6)
    pos = np.column_stack([g.uniform(0, grid.Lx_nm, 50), g.uniform(0, grid.Ly_nm, 50),
                           g.uniform(grid.Lz_nm * 0.1, grid.Lz_nm * 0.9, 50)])
    q = g.normal(size=50)
    rho = charge.deposit(grid, pos, q)
    vol = np.prod(grid.h_m)
    assert abs(rho.sum() * vol - q.sum()) < 1e-12
    phi = g.normal(size=grid.shape)
    assert abs((rho * phi).sum() * vol - (q * charge.gather(grid, phi, pos)).sum()) < 1e-10
    # a node-centred atom gathers exactly the node value
    hx, hy, hz = grid.h_m * 1e9
    p1 = np.array([[2 * hx, 1 * hy, 5 * hz]])
    assert abs(charge.gather(grid, phi, p1)[0] - phi[4, 1, 2]) < 1e-12


def test_host_core_csr_product_is_the_csr_product():
    """The oracle's OpenMP CSR loop computes A x as scipy's product does (same row sums in the
    same order: agreement to rounding), and the thread count changes no bit."""
    from oracle import hamiltonian, spmv
    spec = synth.lattice_spec(3, 4, 5, (0, 1, 0), seed=12, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(12, 10, 2)
    H = hamiltonian.assemble(spec, p).tocsr()
    H.sort_indices()
    x = synth.random_vectors(3, H.shape[0])[0]
    ref = H @ x
    y1 = spmv.matvec(H, x, threads=1)
    y4 = spmv.matvec(H, x, threads=4)
    assert np.array_equal(y1, y4)
    assert np.abs(y1 - ref).max() <= 1e-14 * np.abs(ref).max()
    # a hand-sized case: [[2, 0, 1], [0, 0, 0], [-1, 3, 0]] (1, 2, 3) = (5, 0, 5)
    import scipy.sparse as sp
    A = sp.csr_matrix(np.array([[2.0, 0, 1], [0, 0, 0], [-1, 3, 0]]))
    assert np.array_equal(spmv.matvec(A, np.array([1.0, 2.0, 3.0])), [5.0, 0.0, 5.0])
