"""Pins of the oracle's Euler<->Lagrange coupling operators (Sec. 3.1.2 Eq.
filter_def / Eq. interpolation, Sec. 3.2.1 Eqs. distribution_filter and
fluid_volume_fraction) against properties the mathematics fixes."""
import numpy as np
import pytest

import oracle as O


def test_phi_values_and_continuity():
    # exact values of the three-point function at r = 0, 1/2, 1, 3/2
    assert O.phi(0.0) == pytest.approx(2.0 / 3.0, abs=1e-16)
    assert O.phi(0.5) == pytest.approx(0.5, abs=1e-16)
    assert O.phi(1.0) == pytest.approx(1.0 / 6.0, abs=1e-16)
    assert O.phi(1.5) == 0.0
    assert O.phi(2.0) == 0.0
    # continuity at the branch points
    for r0 in (0.5, 1.5):
        assert abs(O.phi(r0 - 1e-12) - O.phi(r0 + 1e-12)) < 1e-6
    # even function
    for r in np.linspace(0, 1.6, 17):
        assert O.phi(r) == O.phi(-r)


@pytest.mark.parametrize("s", np.linspace(-0.5, 0.5, 41))
def test_phi_moment_identities(s):
    """Partition of unity, zero first moment and sum of squares 1/2 for every
    shift: the defining properties of the three-point delta function."""
    j = np.arange(-3, 4)
    w = np.array([O.phi(jj - s) for jj in j])
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert (w * (j - s)).sum() == pytest.approx(0.0, abs=1e-15)
    assert (w * w).sum() == pytest.approx(0.5, abs=1e-15)


def _params(n, periodic):
    return O.make_params(n, periodic, tau=0.8)


def test_weights_periodic_wrap_and_walls():
    idx, wt = O.weights_1d(0.2, 8, True)
    assert list(idx) == [7, 0, 1]
    assert wt.sum() == pytest.approx(1.0, abs=1e-15)
    idx, wt = O.weights_1d(0.2, 8, False)
    assert idx[0] == -1 and wt[0] == 0.0
    assert wt.sum() == pytest.approx(1.0, abs=1e-15)
    # renormalisation keeps the ratio of the in-domain weights
    assert wt[2] / wt[1] == pytest.approx(O.phi(1.3) / O.phi(0.3), rel=1e-14)


def test_self_interpolated_solid_fraction_is_V_over_8():
    """An isolated particle sees eps_p|p = V/8 dx^3 wherever it sits (tensor
    product of three 1D kernels, each with sum of squares 1/2)."""
    rng = np.random.default_rng(1)
    P = _params((12, 12, 12), (1, 1, 1))
    for _ in range(20):
        x = rng.uniform(0, 12, size=(1, 3))
        d = np.array([0.9])
        eps_p = O.solid_fraction(P, x, d)
        V = np.pi / 6 * 0.9 ** 3
        assert O.interpolate(P, eps_p, x[0])[0] == pytest.approx(V / 8, rel=1e-14)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 1, 0), (0, 0, 0)])
def test_volume_conservation(periodic):
    """sum_x eps_p dx^3 = sum_i V_i (partition of unity, walls renormalised)."""
    rng = np.random.default_rng(2)
    P = _params((10, 9, 11), periodic)
    x = rng.uniform(0.05, 1, size=(200, 3)) * np.array([10, 9, 11])
    d = rng.uniform(0.5, 1.2, size=200)
    eps_p = O.solid_fraction(P, x, d)
    assert eps_p.sum() == pytest.approx((np.pi / 6 * d ** 3).sum(), rel=1e-13)
    eps_f, nclamp = O.fluid_fraction(P, x, d)
    assert nclamp == 0
    np.testing.assert_allclose(eps_f, 1.0 - eps_p, rtol=0, atol=1e-15)


def test_distribution_conserves_momentum_and_first_moment():
    rng = np.random.default_rng(3)
    P = _params((8, 8, 8), (1, 1, 1))
    x = rng.uniform(0, 8, size=(30, 3))
    F = rng.normal(size=(30, 3))
    out = O.distribute(P, x, F, scale=1.0)
    np.testing.assert_allclose(out.sum(axis=1), F.sum(axis=0), rtol=1e-13)
    # a single particle away from the periodic seam: centroid of the spread
    # force density sits exactly at the particle (zero first moment)
    P2 = _params((10, 10, 10), (0, 0, 0))
    xp = np.array([[4.3, 5.71, 3.05]])
    out = O.distribute(P2, xp, np.array([[1.0, 0.0, 0.0]]))
    idx = np.arange(1000)
    centres = np.stack([idx % 10, (idx // 10) % 10, idx // 100], 1) + 0.5
    np.testing.assert_allclose((out[0][:, None] * centres).sum(0), xp[0], rtol=0, atol=1e-13)


def test_interpolation_exact_for_linear_fields():
    """Zero first moment: a linear field is interpolated exactly (interior)."""
    P = _params((10, 10, 10), (0, 0, 0))
    idx = np.arange(1000)
    centres = np.stack([idx % 10, (idx // 10) % 10, idx // 100], 1) + 0.5
    a = np.array([0.3, -1.2, 2.5])
    field = centres @ a + 0.7
    rng = np.random.default_rng(4)
    for _ in range(10):
        xp = rng.uniform(2, 8, size=3)
        assert O.interpolate(P, field, xp)[0] == pytest.approx(xp @ a + 0.7, rel=1e-13)
