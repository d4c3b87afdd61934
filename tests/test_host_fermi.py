"""omen_fermi_level runs on the host only: checked on the CPU against the oracle's bisection
and against the electron count it is defined by (Section III-A item 2: the Fermi level from
charge neutrality)."""
import numpy as np
import pytest

from oracle import charge


@pytest.fixture(scope="module")
def omen():
    from paper_1003_4570_gb300 import build
    build.build()
    from paper_1003_4570_gb300 import omen as om
    return om


@pytest.mark.parametrize("kT,target", [(0.0003447, 13.7), (0.01, 13.7), (0.05, 0.3), (0.025, 39.9)])
def test_fermi_level_matches_the_oracle(omen, kT, target):
    g = np.random.default_rng(11)
    E = np.sort(g.uniform(-1, 1, 40))
    W = g.uniform(0.5, 2, 40) * (target / 13.7 if target > 30 else 1.0)
    if target > W.sum():
        W *= 1.1 * target / W.sum()
    ef = omen.omen_fermi_level(E, W, target, kT)
    assert abs((W * charge.fermi(E, ef, kT)).sum() - target) < 1e-9 * max(1.0, target)
    ref = charge.fermi_level([E], [1.0], target, kT, 1.0) if np.allclose(W, W[0]) else None
    if ref is not None:
        assert abs(ef - ref) < 1e-10


def test_fermi_level_with_equal_weights_equals_the_oracle(omen):
    """Equal level weights w: the oracle's gs * sum over one k set with weight 1 is the same sum."""
    g = np.random.default_rng(12)
    E = np.sort(g.uniform(-2, 1, 64))
    for kT, target in ((0.0003447, 17.0), (0.02, 9.25)):
        ef = omen.omen_fermi_level(E, np.full(64, 2.0), target, kT)
        ref = charge.fermi_level([E], [1.0], target, kT, 2.0)
        assert abs(ef - ref) < 1e-10


def test_degenerate_levels_and_unreachable_targets(omen):
    E = np.array([-0.5, -0.5, -0.5, 0.2, 0.2])
    W = np.ones(5)
    # three equal levels hold 1.5 electrons at E_F = -0.5 exactly (each half full)
    ef = omen.omen_fermi_level(E, W, 1.5, 0.01)
    assert abs(ef + 0.5) < 1e-9
    for bad in (-1.0, 5.0 + 1e-9, 6.0):
        with pytest.raises(omen.OmenError):
            omen.omen_fermi_level(E, W, bad, 0.01)
    # the limits (empty, full) are met outside the levels, to rounding of the count
    for target, side in ((0.0, -1), (5.0, 1)):
        ef = omen.omen_fermi_level(E, W, target, 0.01)
        assert side * (ef - (0.2 if side > 0 else -0.5)) > 10 * 0.01
        assert abs((W * charge.fermi(E, ef, 0.01)).sum() - target) < 1e-12
