"""The seeded input generators: deterministic per seed, the documented ranges and layouts."""
import numpy as np

import synth


def test_same_seed_same_inputs_and_streams_independent():
    a = synth.lattice_spec(3, 3, 3, (1, 1, 0), seed=5, alloy_fraction=0.3, strain_amp=0.02)
    b = synth.lattice_spec(3, 3, 3, (1, 1, 0), seed=5, alloy_fraction=0.3, strain_amp=0.02)
    c = synth.lattice_spec(3, 3, 3, (1, 1, 0), seed=6, alloy_fraction=0.3, strain_amp=0.02)
    assert np.array_equal(a.species, b.species) and np.array_equal(a.strain, b.strain)
    assert not np.array_equal(a.species, c.species)
    # strain draws do not depend on whether species were drawn (separate streams)
    d = synth.lattice_spec(3, 3, 3, (1, 1, 0), seed=5, alloy_fraction=0.0, strain_amp=0.02)
    assert np.array_equal(a.strain, d.strain)


def test_documented_ranges():
    s = synth.lattice_spec(20, 20, 20, (0, 0, 0), seed=1, alloy_fraction=0.3, strain_amp=0.02)
    assert s.species.dtype == np.uint8 and s.species.shape == (8 * 8000,)
    assert abs(s.species.mean() - 0.3) < 0.01
    assert s.strain.shape == (16 * 8000,) and np.abs(s.strain).max() <= 0.02
    p = synth.draw_tb_params(3, synth.SP3D5S, 2)
    assert p.V.shape == (2, 2, 14) and np.all(np.abs(p.V) <= 3.0)
    e = synth.effmass_spec(4, 5, 6, seed=2, u_amp=0.1)
    assert e.U.shape == (120,) and np.abs(e.U).max() <= 0.1 and e.npoints == 120
    v = synth.draw_vff_params(4)
    ev_per_nm2 = synth.N_PER_M_IN_EV_PER_NM2
    assert np.all((v.alpha >= 38 * ev_per_nm2) & (v.alpha <= 50 * ev_per_nm2))
    assert np.all((v.beta >= 10 * ev_per_nm2) & (v.beta <= 15 * ev_per_nm2))
    assert abs(ev_per_nm2 - 6.241509074) < 1e-8


def test_doping_draws():
    for seed in range(20):
        ns, w = synth.draw_doping(seed)
        assert 1e13 <= ns <= 2e14 and 0.5 <= w <= 2.0
