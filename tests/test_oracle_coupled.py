"""Pins of the oracle's coupled step (Algorithm 1) against global balances and
the single-sphere closed forms."""
import math

import numpy as np
import pytest

import oracle as O

C, W, _ = O.lattice()


def _fluid_momentum(dom):
    rho, j = O.moments(dom.P, dom.f)
    return j.sum(axis=1)


def _particle_momentum(dom):
    n = dom.np
    m = dom.rho_p[:n] * math.pi / 6 * dom.d[:n] ** 3
    return (m[:, None] * dom.u[:n]).sum(0)


def test_total_momentum_conserved_without_pressure_force():
    """Periodic box, gravity on the particles balanced by eps_f f_b on the
    fluid, pressure-gradient force off: drag and added-mass reactions and the
    pair forces exchange momentum exactly, so fluid + particle momentum is
    constant to round-off over several coupled steps with subcycling."""
    rng = np.random.default_rng(21)
    n = (8, 8, 8)
    npart = 24
    x = rng.uniform(0, 8, size=(npart, 3))
    d = np.full(npart, 0.9)
    rho_p = np.full(npart, 2.5)
    g = np.array([0.0, 0.0, -4e-3])
    V = math.pi / 6 * d ** 3
    f_b = -((rho_p - 1.0) * V).sum() * g / (np.prod(n) - V.sum())
    P = O.make_params(n, (1, 1, 1), tau=0.7, g=g, f_b=f_b, n_int=2, n_dem=4, pressure=0,
                      h_c=0.9, T_c=1.0, e_n=0.9)
    dom = O.Domain(P, x=x, u=0.01 * rng.standard_normal((npart, 3)), d=d, rho_p=rho_p)
    tot0 = _fluid_momentum(dom) + _particle_momentum(dom)
    for _ in range(6):
        dom.step(1)
        tot = _fluid_momentum(dom) + _particle_momentum(dom)
        np.testing.assert_allclose(tot, tot0, atol=1e-14)
    assert dom.counters["eps_clamp"] == 0
    # the exchange is not trivial: the fluid has picked up momentum
    assert np.abs(_fluid_momentum(dom)).max() > 1e-4


def test_fluid_gains_exactly_the_applied_force_density():
    """One step with the pressure force on: the fluid momentum changes by the
    sum of f_ext = f_pf + eps_f f_b actually applied (Guo scheme)."""
    rng = np.random.default_rng(22)
    n = (8, 8, 8)
    x = rng.uniform(0, 8, size=(10, 3))
    P = O.make_params(n, (1, 1, 1), tau=0.8, g=(0, 0, -3e-3), f_b=(0, 0, 1e-5), n_int=3, n_dem=2)
    dom = O.Domain(P, x=x, d=np.full(10, 1.0), rho_p=np.full(10, 2.5))
    dom.step(2)
    j0 = _fluid_momentum(dom)
    dom.step(1)
    fx = dom.fields()["f_ext"].sum(axis=1)
    np.testing.assert_allclose(_fluid_momentum(dom) - j0, fx, rtol=1e-12, atol=1e-14)


def test_single_sphere_terminal_velocity_and_force_balance():
    """Single settling sphere in a walled box: at terminal velocity the frozen
    hydrodynamic force balances the buoyant weight, and the velocity is of the
    Stokes magnitude u_St = (rho_p - rho_f) g d^2 / (18 mu)."""
    tau = 0.65
    mu = (tau - 0.5) / 3
    d = 0.8
    u_st = 0.1 * mu / d  # Re_p = 0.1
    g = 18 * mu * u_st / (1.5 * d * d)
    P = O.make_params((16, 16, 32), (1, 1, 0), tau=tau, g=(0, 0, -g), h_c=d, T_c=1.0)
    dom = O.Domain(P, x=[[8.0, 8.0, 24.0]], d=[d], rho_p=[2.5])
    dom.step(500)
    w = 1.5 * math.pi / 6 * d ** 3 * g
    # steady: net force (hydrodynamic + gravity) small against the weight
    assert abs(dom.F_hyd[0, 2]) < 2e-3 * w
    ratio = -dom.u[0, 2] / u_st
    assert 0.5 < ratio < 1.5
    assert abs(dom.u[0, 0]) < 1e-12 and abs(dom.u[0, 1]) < 1e-12
