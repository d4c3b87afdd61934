"""Warm-start network on the GPU against the oracle, and what it gains the SCF loop.

* forward outputs, loss gradients and one Adam step equal the FP64 oracle evaluated with the
  same BF16-rounded weights (tolerances from FP32 accumulation: 1e-5 relative for outputs,
  1e-3 of each layer's largest gradient, 1e-6 for the updated weights);
* feature / target / warm-start maps equal the oracle maps;
* trained on self-consistent potentials that omen_scf produces for seeded delta-doping
  profiles, the network's start needs fewer SCF iterations than the zero-field start on held-out
  profiles, and both starts converge to the same potential (1e-6 V tolerance of the loop);
* a start that is far off falls back to the zero-field start (omen_scf_learned).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp as omlp, poisson  # noqa: E402

SIZES = (256, 512, 512, 256)


@pytest.fixture(scope="module")
def ctx():
    from paper_1003_4570_gb300 import omen
    return omen.omen_create(0, torch.cuda.current_stream().cuda_stream)


def test_forward_gradients_adam_match_oracle(ctx):
    from paper_1003_4570_gb300 import omen
    p0 = synth.mlp_init(5, SIZES)
    net = omen.omen_mlp_create(ctx, p0)
    w16 = omen.omen_mlp_get_params(ctx, net, bf16_rounded=True).astype(float)
    np.testing.assert_array_equal(w16[: SIZES[1] * SIZES[0]], omlp.bf16_round(p0[: SIZES[1] * SIZES[0]]))
    g = np.random.default_rng(0)
    B = 37
    X = g.normal(size=(B, SIZES[0])).astype(np.float32)
    T = g.normal(size=(B, SIZES[3])).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Yd = torch.empty((B, SIZES[3]), dtype=torch.float32, device="cuda")
    omen.omen_mlp_forward(ctx, net, Xd, B, Yd)
    torch.cuda.synchronize()
    _, _, Yref = omlp.forward(w16, SIZES, X.astype(float))
    np.testing.assert_allclose(Yd.cpu().numpy(), Yref, atol=1e-5 * np.abs(Yref).max(), rtol=0)
    grad, loss = omen.omen_mlp_gradients(ctx, net, Xd, Td, B)
    loss_ref, grad_ref = omlp.loss_and_grads(w16, SIZES, X.astype(float), T.astype(float))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    off = 0
    for l in range(3):
        for n in (SIZES[l + 1] * SIZES[l], SIZES[l + 1]):
            seg = slice(off, off + n)
            np.testing.assert_allclose(grad[seg], grad_ref[seg], atol=1e-3 * np.abs(grad_ref[seg]).max(), rtol=0)
            off += n
    omen.omen_mlp_train_step(ctx, net, Xd, Td, B, lr=1e-3)
    w1 = omen.omen_mlp_get_params(ctx, net)
    w1_ref, _, _ = omlp.adam_step(p0.astype(float), 0.0, 0.0, grad.astype(float), 1, 1e-3)
    np.testing.assert_allclose(w1, w1_ref, atol=1e-6, rtol=0)


def test_profile_maps_match_oracle(ctx):
    from paper_1003_4570_gb300 import omen
    net = omen.omen_mlp_create(ctx, synth.mlp_init(6, SIZES))
    grid = poisson.Grid(3, 3, 217, 2.1724, 2.1724, 43.448)
    rho = synth.donor_rho_on_grid(6.3e13, 1.3, grid.nx, grid.ny, grid.nz, grid.Lz_nm)
    x = torch.empty(256, dtype=torch.float32, device="cuda")
    omen.omen_mlp_features(ctx, net, grid, torch.from_numpy(rho).cuda(), x)
    torch.cuda.synchronize()
    np.testing.assert_allclose(x.cpu().numpy(), omlp.features(grid, rho), atol=2e-6)
    phi = np.random.default_rng(1).normal(size=grid.shape) * 0.05
    t = torch.empty(256, dtype=torch.float32, device="cuda")
    omen.omen_mlp_targets(ctx, net, grid, torch.from_numpy(phi).cuda(), t)
    torch.cuda.synchronize()
    np.testing.assert_allclose(t.cpu().numpy(), omlp.targets(grid, phi), atol=2e-6)
    ws = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
    omen.omen_mlp_warm_start(ctx, net, grid, torch.from_numpy(rho).cuda(), ws)
    torch.cuda.synchronize()
    w16 = omen.omen_mlp_get_params(ctx, net, bf16_rounded=True).astype(float)
    _, _, y = omlp.forward(w16, SIZES, omlp.features(grid, rho)[None, :])
    np.testing.assert_allclose(ws.cpu().numpy(), omlp.inject(grid, y[0]), atol=1e-5)


def delta_problem(seed, nzc=16):
    spec, p, _ = synth.delta_layer(1, nzc, seed=1)
    a = spec.a_nm
    grid = poisson.Grid(3, 3, round(nzc * a / 0.2), a, a, nzc * a)
    ns, w = synth.draw_doping(seed)
    rho = synth.donor_rho_on_grid(ns, w, grid.nx, grid.ny, grid.nz, grid.Lz_nm)
    eg = synth.GAPPED_SI_EC - synth.GAPPED_SI_EV
    kw = dict(n_electrons=ns * (a * 1e-7) ** 2, kT=8.617333262e-5 * 4, kpts=[(0.0, 0.0, 0.0)], kweights=[1.0],
              nev=8, sigma=synth.GAPPED_SI_EC - 0.4 * eg, e_cut=0.5 * (synth.GAPPED_SI_EC + synth.GAPPED_SI_EV))
    return spec, p, grid, rho, kw


def run_scf(omen, ctx, lat, p, grid, rho_d, phi, kw):
    return omen.omen_scf(ctx, lat, p, grid, phi, rho_d, eig_tol=1e-10, eig_block=1, eig_basis=48, mix=0.3,
                         mix_history=6, tol_V=1e-6, max_iter=200, **kw)


def test_learned_start_saves_scf_iterations(ctx):
    from paper_1003_4570_gb300 import omen
    n_train, n_test = 16, 3
    spec, p, grid, _, _ = delta_problem(0)
    lat = omen.omen_build_lattice(ctx, spec)
    net = omen.omen_mlp_create(ctx, synth.mlp_init(7, SIZES))
    X = torch.empty((n_train, 256), dtype=torch.float32, device="cuda")
    T = torch.empty((n_train, 256), dtype=torch.float32, device="cuda")
    for i in range(n_train):
        _, _, _, rho, kw = delta_problem(1000 + i)
        rho_d = torch.from_numpy(rho).cuda()
        phi = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        info, _ = run_scf(omen, ctx, lat, p, grid, rho_d, phi, kw)
        assert info["converged"] == 1
        omen.omen_mlp_features(ctx, net, grid, rho_d, X[i])
        omen.omen_mlp_targets(ctx, net, grid, phi, T[i])
    for _ in range(400):
        loss = omen.omen_mlp_train_step(ctx, net, X, T, n_train, lr=1e-3)
    assert loss < 1e-2
    saved = []
    for i in range(n_test):
        _, _, _, rho, kw = delta_problem(5000 + i)
        rho_d = torch.from_numpy(rho).cuda()
        phi0 = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        info0, _ = run_scf(omen, ctx, lat, p, grid, rho_d, phi0, kw)
        phi1 = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
        omen.omen_mlp_warm_start(ctx, net, grid, rho_d, phi1)
        info1, _ = run_scf(omen, ctx, lat, p, grid, rho_d, phi1, kw)
        assert info0["converged"] == 1 and info1["converged"] == 1
        # both are fixed points within the loop tolerance: their difference is a few tol_V
        assert (phi0 - phi1).abs().max().item() < 1e-5
        saved.append(info0["iterations"] - info1["iterations"])
    # at least one iteration saved on average, and no held-out profile worse off
    assert np.mean(saved) >= 1 and min(saved) >= 0, saved


def test_learned_start_falls_back_to_zero_field(ctx):
    """A network whose output is far off (an output bias of 50, i.e. 10 V everywhere) cannot reach
    the fixed point within the iteration budget that suffices from zero field: omen_scf_learned
    then starts again from zero field, and returns that run's potential, the same as a plain
    zero-field solve."""
    from paper_1003_4570_gb300 import omen
    spec, p, grid, rho, kw = delta_problem(4242)
    lat = omen.omen_build_lattice(ctx, spec)
    params = synth.mlp_init(7, SIZES).copy()
    params[-SIZES[3]:] = 50.0
    net = omen.omen_mlp_create(ctx, params)
    rho_d = torch.from_numpy(rho).cuda()
    phi0 = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    info0, _ = run_scf(omen, ctx, lat, p, grid, rho_d, phi0, kw)
    assert info0["converged"] == 1 and info0["iterations"] < 40
    phi1 = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
    info1, st, fallback = omen.omen_scf_learned(ctx, net, lat, p, grid, phi1, rho_d, eig_tol=1e-10, eig_block=1,
                                                eig_basis=48, mix=0.3, mix_history=6, tol_V=1e-6, max_iter=40, **kw)
    assert fallback and info1["converged"] == 1
    assert abs(info1["iterations"] - info0["iterations"]) <= 1
    # the same loop from the same start (the charge deposit sums atoms in no fixed order, so the
    # two runs agree to rounding, well inside the loop tolerance)
    assert (phi0 - phi1).abs().max().item() < 1e-7
    # a good start needs no fallback
    good = omen.omen_mlp_create(ctx, synth.mlp_init(7, SIZES) * 0.0)
    phi2 = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
    _, _, fb2 = omen.omen_scf_learned(ctx, good, lat, p, grid, phi2, rho_d, eig_tol=1e-10, eig_block=1, eig_basis=48,
                                      mix=0.3, mix_history=6, tol_V=1e-6, max_iter=40, **kw)
    assert not fb2
