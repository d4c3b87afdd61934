"""H·X parity: the CUDA product against the oracle's explicit CSR, element by element.

Sizes span several 128-thread tiles with a ragged tail (cells not a multiple of 128);
boundaries hard wall / periodic / Bloch; sp3s* and sp3d5s*; spin-orbit; stored and
matrix-free; FP64 and FP32.  Tolerances: FP64 1e-12 of max|y|; FP32 2e-6 of max|y|
(float rounding of blocks and vectors over ~50 terms per row).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import hamiltonian  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1003_4570_gb300 import omen
    return omen.omen_create(0, torch.cuda.current_stream().cuda_stream)


CASES = [
    # (dims, periodic, basis, nspecies, alloy, strain, so, k, precision, matrix_free)
    ((5, 4, 7), (0, 0, 0), 10, 2, 0.3, 0.02, False, None, 0, False),
    ((5, 4, 7), (1, 1, 1), 5, 1, 0.0, 0.0, False, None, 0, False),
    ((3, 6, 9), (1, 0, 1), 10, 2, 0.5, 0.02, False, None, 0, True),
    ((4, 3, 11), (2, 2, 0), 10, 2, 0.3, 0.02, False, (0.31, -0.52, 0.0), 0, False),
    ((4, 3, 11), (2, 2, 0), 10, 2, 0.3, 0.02, False, (0.31, -0.52, 0.0), 0, True),
    ((3, 5, 9), (0, 1, 0), 10, 2, 0.3, 0.02, True, None, 0, False),
    ((3, 5, 9), (2, 1, 0), 5, 2, 0.3, 0.02, True, (0.7, 0.0, 0.0), 0, True),
    ((5, 4, 7), (0, 0, 0), 10, 2, 0.3, 0.02, False, None, 1, False),
    ((3, 5, 9), (0, 1, 0), 10, 2, 0.3, 0.02, True, None, 1, False),
    ((4, 3, 11), (2, 2, 0), 10, 2, 0.3, 0.02, False, (0.31, -0.52, 0.0), 1, True),
    # one-cell periodic directions (every lateral bond reaches a periodic image of the same cell)
    ((1, 1, 6), (2, 2, 0), 10, 2, 0.3, 0.02, False, (1.1, -0.7, 0.0), 0, False),
    ((1, 1, 1), (1, 1, 1), 5, 1, 0.0, 0.0, False, None, 0, False),
    ((1, 2, 1), (0, 1, 2), 10, 2, 0.5, 0.02, True, (0.0, 0.0, 0.9), 1, False),
]


@pytest.mark.parametrize("case", CASES, ids=[f"c{i}" for i in range(len(CASES))])
def test_hx_matches_oracle(ctx, case):
    from paper_1003_4570_gb300 import omen
    dims, per, basis, ns, alloy, strain, so, k, prec, mf = case
    spec = synth.lattice_spec(*dims, per, seed=31, alloy_fraction=alloy, strain_amp=strain)
    p = synth.draw_tb_params(31, basis, ns)
    U = np.random.default_rng(2).uniform(-0.2, 0.2, spec.natoms)
    H = hamiltonian.assemble(spec, p, U_atom=U, kvec=k, spin_orbit=so)
    lat = omen.omen_build_lattice(ctx, spec)
    n_atoms, n_bonds = lat.counts()
    assert n_atoms == spec.natoms
    Ud = torch.from_numpy(U).cuda()
    ham = omen.omen_assemble_H(ctx, lat, p, spin_orbit=so, precision=prec, matrix_free=mf, k=k, U_atom_dev=Ud)
    assert ham.nrows == H.shape[0]
    sigma = 0.37
    x = synth.random_vectors(5, H.shape[0], 2, dtype=complex if ham.is_complex else float)
    xd = torch.from_numpy(x.astype(ham.numpy_dtype)).cuda()
    yd = torch.empty_like(xd)
    omen.omen_hx(ctx, ham, xd, yd, nvec=2, sigma=sigma)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    for v in range(2):
        xv = x[v].astype(ham.numpy_dtype).astype(complex if ham.is_complex else float)
        ref = H @ xv - sigma * xv
        scale = np.abs(ref).max()
        tol = 1e-12 if prec == 0 else 2e-6
        np.testing.assert_allclose(y[v], ref, atol=tol * scale, rtol=0)


def test_hx_host_entry_point(ctx):
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(3, 3, 3, (0, 1, 0), seed=8, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(8, 10, 2)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p)
    H = hamiltonian.assemble(spec, p)
    x = synth.random_vectors(9, H.shape[0], 3)
    y = omen.omen_hx_host(ctx, ham, x, sigma=-0.5)
    for v in range(3):
        ref = H @ x[v] + 0.5 * x[v]
        np.testing.assert_allclose(y[v], ref, atol=1e-12 * np.abs(ref).max(), rtol=0)


def test_hard_wall_bond_count_and_invalid_species(ctx):
    from paper_1003_4570_gb300 import omen
    for n in (1, 2, 5):
        spec = synth.lattice_spec(n, n, n, (0, 0, 0))
        lat = omen.omen_build_lattice(ctx, spec)
        assert lat.counts() == (8 * n ** 3, 16 * n ** 3 - 12 * n ** 2 + 3 * n)
    spec = synth.lattice_spec(2, 2, 2, (1, 1, 1), alloy_fraction=0.5, seed=3)
    lat = omen.omen_build_lattice(ctx, spec)
    p = synth.draw_tb_params(3, 5, 1)  # one species, but the structure has two
    with pytest.raises(omen.OmenError) as e:
        omen.omen_assemble_H(ctx, lat, p)
    assert e.value.status == omen.OMEN_EINVAL


def test_double_float_hx_matches_oracle(ctx):
    """OMEN_F64_DF: FP64-accurate product on the FP32 pipe, same 1e-12 tolerance as FP64."""
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(5, 4, 7, (0, 1, 0), seed=33, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(33, 10, 2)
    U = np.random.default_rng(4).uniform(-0.2, 0.2, spec.natoms)
    H = hamiltonian.assemble(spec, p, U_atom=U)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p, precision=omen.OMEN_F64_DF, U_atom_dev=torch.from_numpy(U).cuda())
    x = synth.random_vectors(6, H.shape[0], 2)
    y = omen.omen_hx_host(ctx, ham, x, sigma=0.21)
    for v in range(2):
        ref = H @ x[v] - 0.21 * x[v]
        np.testing.assert_allclose(y[v], ref, atol=1e-12 * np.abs(ref).max(), rtol=0)
    # device buffers in double-float form
    n = H.shape[0]
    xd = torch.from_numpy(x[0]).cuda()
    xdf = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    ydf = torch.empty_like(xdf)
    yd = torch.empty(n, dtype=torch.float64, device="cuda")
    from paper_1003_4570_gb300.omen import lib
    ctx.check(lib().omen_convert_vectors(ctx.handle, xd.data_ptr(), omen.OMEN_F64, xdf.data_ptr(), omen.OMEN_F64_DF, n))
    omen.omen_hx(ctx, ham, xdf, ydf, 1, 0.0)
    ctx.check(lib().omen_convert_vectors(ctx.handle, ydf.data_ptr(), omen.OMEN_F64_DF, yd.data_ptr(), omen.OMEN_F64, n))
    torch.cuda.synchronize()
    ref = H @ x[0]
    np.testing.assert_allclose(yd.cpu().numpy(), ref, atol=1e-12 * np.abs(ref).max(), rtol=0)
    with pytest.raises(omen.OmenError) as e:
        omen.omen_assemble_H(ctx, lat, p, precision=omen.OMEN_F64_DF, spin_orbit=True)
    assert e.value.status == omen.OMEN_EUNSUPPORTED


TILE_CASES = [
    # (dims, periodic, basis, so, k, precision, matrix_free)
    ((5, 4, 7), (0, 0, 0), 10, False, None, 1, False),
    ((5, 4, 7), (0, 1, 0), 10, False, None, 0, False),
    ((3, 5, 9), (0, 1, 0), 10, True, None, 1, False),
    ((4, 3, 11), (1, 1, 0), 5, False, None, 1, False),
    ((4, 3, 11), (2, 2, 0), 10, False, (0.31, -0.52, 0.0), 1, True),
]


@pytest.mark.parametrize("case", TILE_CASES, ids=[f"t{i}" for i in range(len(TILE_CASES))])
def test_every_launch_shape_gives_the_same_product(ctx, case):
    """Each compiled (CTA width, rows per register batch) gives the default shape's result bit
    for bit (same summation order per accumulator), and that result matches the oracle."""
    from paper_1003_4570_gb300 import omen
    dims, per, basis, so, k, prec, mf = case
    spec = synth.lattice_spec(*dims, per, seed=35, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(35, basis, 2)
    H = hamiltonian.assemble(spec, p, kvec=k, spin_orbit=so)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p, spin_orbit=so, precision=prec, matrix_free=mf, k=k)
    x = synth.random_vectors(7, H.shape[0], 2, dtype=complex if ham.is_complex else float)
    xd = torch.from_numpy(x.astype(ham.numpy_dtype)).cuda()

    def product():
        yd = torch.empty_like(xd)
        omen.omen_hx(ctx, ham, xd, yd, nvec=2, sigma=0.2)
        torch.cuda.synchronize()
        return yd.cpu().numpy()

    base = product()
    for v in range(2):
        xv = x[v].astype(ham.numpy_dtype).astype(complex if ham.is_complex else float)
        ref = H @ xv - 0.2 * xv
        tol = 1e-12 if prec == 0 else 2e-6
        np.testing.assert_allclose(base[v], ref, atol=tol * np.abs(ref).max(), rtol=0)
    shapes = 0
    for thr in (32, 64, 96, 128, 256):
        for rb in (0, 1, 2, 5, 10):
            try:
                omen.omen_hx_set_tile(ctx, ham, prec, thr, rb)
            except omen.OmenError as e:
                assert e.status == omen.OMEN_EINVAL
                continue
            shapes += 1
            assert np.array_equal(product(), base), (thr, rb)
    assert shapes >= 4
    for bad in ((48, 0), (256, 0), (128, 3), (128, 7)):
        with pytest.raises(omen.OmenError) as e:
            omen.omen_hx_set_tile(ctx, ham, prec, *bad)
        assert e.value.status == omen.OMEN_EINVAL
    r = omen.omen_tune_hx(ctx, ham, prec, nvec=2, reps=3)
    assert r["candidates"] >= shapes // 2 and r["ms_best"] <= r["ms_default"] + 1e-9
    assert np.array_equal(product(), base)


@pytest.mark.parametrize("prec", [0, 1])
def test_every_kbatch_launch_shape_gives_the_same_product(ctx, prec):
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(3, 2, 9, (2, 2, 0), seed=36, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(36, 10, 2)
    lat = omen.omen_build_lattice(ctx, spec)
    kpts = np.array([[0.1 * q, -0.05 * q, 0.0] for q in range(7)])
    ham = omen.omen_assemble_H(ctx, lat, p, precision=prec, k=(0.0, 0.0, 0.0))
    n = ham.nrows
    x = synth.random_vectors(8, n, len(kpts), dtype=complex)
    xd = torch.from_numpy(x.astype(ham.numpy_dtype)).cuda()

    def product():
        yd = torch.empty_like(xd)
        omen.omen_hx_kbatch(ctx, ham, kpts, xd, yd, sigma=0.1)
        torch.cuda.synchronize()
        return yd.cpu().numpy()

    base = product()
    for q in (0, 6):
        H = hamiltonian.assemble(spec, p, kvec=kpts[q])
        xv = x[q].astype(ham.numpy_dtype).astype(complex)
        ref = H @ xv - 0.1 * xv
        tol = 1e-12 if prec == 0 else 2e-6
        np.testing.assert_allclose(base[q], ref, atol=tol * np.abs(ref).max(), rtol=0)
    for thr in (32, 64, 128):
        for kb in (1, 2, 4):
            if prec == 0 and kb == 4:
                with pytest.raises(omen.OmenError):
                    omen.omen_hx_kbatch_set_tile(ctx, ham, prec, thr, kb)
                continue
            omen.omen_hx_kbatch_set_tile(ctx, ham, prec, thr, kb)
            assert np.array_equal(product(), base), (thr, kb)
    r = omen.omen_tune_hx_kbatch(ctx, ham, len(kpts), reps=3)
    assert r["ms_best"] <= r["ms_default"] + 1e-9
    assert np.array_equal(product(), base)


@pytest.mark.parametrize("per", [(0, 1, 0), (1, 0, 1), (2, 2, 1)])
def test_hx_host_overlapped_slabs(ctx, per):
    """The host-buffer product cuts the structure into z-slabs and overlaps their copies with the
    product: every row must still equal the oracle's (hard-wall and periodic z, 2 vectors)."""
    from paper_1003_4570_gb300 import omen
    spec = synth.lattice_spec(3, 2, 13, per, seed=37, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(37, 10, 2)
    k = (0.2, -0.3, 0.1) if 2 in per else None
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p, k=k)
    H = hamiltonian.assemble(spec, p, kvec=k)
    x = synth.random_vectors(12, H.shape[0], 2, dtype=complex if ham.is_complex else float)
    y = omen.omen_hx_host(ctx, ham, x, sigma=0.3)
    for v in range(2):
        ref = H @ x[v] - 0.3 * x[v]
        np.testing.assert_allclose(y[v], ref, atol=1e-12 * np.abs(ref).max(), rtol=0)
    xp = torch.from_numpy(x).pin_memory()
    yp = torch.empty_like(xp).pin_memory()
    from paper_1003_4570_gb300.omen import lib
    ctx.check(lib().omen_hx_host(ctx.handle, ham.handle, xp.data_ptr(), yp.data_ptr(), 2, 0.3))
    assert np.array_equal(yp.numpy(), y)


def test_fp64_rate_probe(ctx):
    """The FP64 FMA-rate probe the roofline uses returns a plausible device rate (GB300's nominal
    FP64 rate is 1.25 TFLOP/s; a probe outside 0.1-5 TFLOP/s would mean the timing is broken)."""
    from paper_1003_4570_gb300 import omen
    r = omen.omen_probe_fp64_rate(ctx)
    assert 0.1 < r < 5.0, r
