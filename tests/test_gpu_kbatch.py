"""k-batched H·X and lockstep eigen-solves against the oracle, per wave vector.

A strained alloy slab, Bloch-periodic in x and y, hard walls in z; wave vectors along
Gamma-X (and one off-axis).  The batched product must equal the oracle's H(k) x for every k
(FP64 1e-12, FP32 2e-6 of max |y|); the lockstep solver must give each k's lowest
eigenvalues (and the ones nearest sigma, folded) within 1e-9 eV of a dense eigensolve.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import eigs, hamiltonian  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1003_4570_gb300 import omen
    return omen.omen_create(0, torch.cuda.current_stream().cuda_stream)


def slab(nx=3, ny=2, nz=5, seed=51):
    spec = synth.lattice_spec(nx, ny, nz, (2, 2, 0), seed=seed, alloy_fraction=0.3, strain_amp=0.02)
    return spec, synth.draw_tb_params(seed, 10, 2)


def kpath(spec, nk):
    Lx = spec.nx * spec.a_nm
    t = np.linspace(0.07, 0.93, nk)
    k = np.zeros((nk, 3))
    k[:, 0] = t * np.pi / Lx
    k[-1, 1] = 0.4 * np.pi / (spec.ny * spec.a_nm)
    return k


@pytest.mark.parametrize("prec", [0, 1])
def test_hx_kbatch_matches_oracle(ctx, prec):
    from paper_1003_4570_gb300 import omen
    spec, p = slab()
    U = np.random.default_rng(3).uniform(-0.1, 0.1, spec.natoms)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p, precision=prec, k=(0.0, 0.0, 0.0), U_atom_dev=torch.from_numpy(U).cuda())
    ks = kpath(spec, 7)
    x = synth.random_vectors(4, ham.nrows, len(ks), dtype=complex)
    xd = torch.from_numpy(x.astype(ham.numpy_dtype)).cuda()
    yd = torch.empty_like(xd)
    omen.omen_hx_kbatch(ctx, ham, ks, xd, yd, sigma=0.25)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    for q, kv in enumerate(ks):
        H = hamiltonian.assemble(spec, p, U_atom=U, kvec=kv)
        xv = x[q].astype(ham.numpy_dtype).astype(complex)
        ref = H @ xv - 0.25 * xv
        tol = 1e-12 if prec == 0 else 2e-6
        np.testing.assert_allclose(y[q], ref, atol=tol * np.abs(ref).max(), rtol=0)


def test_eigs_kbatch_lowest_and_folded(ctx):
    from paper_1003_4570_gb300 import omen
    spec, p = slab(2, 2, 3, seed=52)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p, k=(0.0, 0.0, 0.0))
    ks = kpath(spec, 5)
    dense = [np.linalg.eigvalsh(hamiltonian.assemble(spec, p, kvec=kv).toarray()) for kv in ks]
    ev, info, st = omen.omen_eigs_kbatch(ctx, ham, ks, 4, tol=1e-9, max_iter=5000, basis=48)
    assert info["converged"] == 1, info
    for q in range(len(ks)):
        np.testing.assert_allclose(ev[q], dense[q][:4], atol=1e-9, rtol=0)
    w0 = dense[0]
    sigma = round(0.5 * (w0[0] + w0[-1]) + 0.3, 3)
    ev, info, st = omen.omen_eigs_kbatch(ctx, ham, ks, 4, which=omen.OMEN_NEAREST, sigma=sigma, tol=1e-7,
                                         max_iter=60000, basis=64)
    assert info["converged"] == 1, info
    for q in range(len(ks)):
        np.testing.assert_allclose(ev[q], eigs.nearest(dense[q], sigma, 4), atol=1e-9, rtol=0)
