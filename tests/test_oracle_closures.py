"""Pins of the oracle's optional closures (the paper's sensitivity models):
the lattice curl (Sec. 3.2.3), the shear lift force (Table 1), the modified
viscosity of Eilers (Eq. visc_eilers) and the Smagorinsky relaxation time
(Eqs. visc_turb, tau_t, tau_e)."""
import math

import numpy as np
import pytest

import oracle as O

C, W, _ = O.lattice()
CS2 = 1.0 / 3.0


def test_curl_exact_on_linear_fields_interior():
    n = (7, 8, 6)
    P = O.make_params(n, (0, 0, 0), tau=0.8)
    idx = np.arange(O.ncell(P))
    X = np.stack([idx % 7, (idx // 7) % 8, idx // 56], 1).astype(float)
    A = np.array([[0.3, -1.1, 0.7], [2.0, 0.4, -0.5], [0.9, 1.3, -0.2]])
    psi = (X @ A.T).T  # psi_a = A_ab x_b
    cu = O.lattice_curl(P, psi)
    expect = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    inner = (X[:, 0] > 0) & (X[:, 0] < 6) & (X[:, 1] > 0) & (X[:, 1] < 7) & (X[:, 2] > 0) & (X[:, 2] < 5)
    for a in range(3):
        np.testing.assert_allclose(cu[a][inner], expect[a], rtol=1e-13)


def test_curl_of_periodic_shear_wave():
    """psi = (0, sin(kx), 0): (curl psi)_z = d_x psi_y = sin(k) cos(kx) on D3Q19."""
    L = 10
    P = O.make_params((L, 4, 5), (1, 1, 1), tau=0.8)
    idx = np.arange(O.ncell(P))
    ix = idx % L
    k = 2 * math.pi / L
    psi = np.zeros((3, O.ncell(P)))
    psi[1] = np.sin(k * ix)
    cu = O.lattice_curl(P, psi)
    np.testing.assert_allclose(cu[2], math.sin(k) * np.cos(k * ix), atol=1e-14)
    np.testing.assert_allclose(cu[:2], 0, atol=1e-14)


def test_lift_is_saffman_and_points_to_the_faster_fluid():
    """Saffman (1965): |F| = 6.46 mu a^2 |du| sqrt(|w|/nu) for du perpendicular
    to w; the paper's 1.61 d^2 sqrt(mu rho/|w|) |du x w| is the same law (1.61 ~
    6.46/4); a sphere lagging a shear flow moves towards the faster fluid."""
    mu, rho, d = 0.05, 1.0, 0.8
    U, gam = 0.01, 0.003
    du = np.array([U, 0, 0])      # fluid faster than the particle along x
    w = np.array([0, 0, -gam])    # vorticity of u_x increasing with y
    F = O.lift(d, mu, rho, du, w)
    saffman = 6.46 * mu * (d / 2) ** 2 * U * math.sqrt(gam / (mu / rho))
    assert np.linalg.norm(F) == pytest.approx(saffman * 1.61 / 1.615, rel=1e-12)
    assert F[1] > 0 and abs(F[0]) < 1e-18 and abs(F[2]) < 1e-18
    assert np.allclose(O.lift(d, mu, rho, du, np.zeros(3)), 0)
    # perpendicular to both du and w for any orientation
    rng = np.random.default_rng(3)
    for _ in range(5):
        a, b = rng.normal(size=3), rng.normal(size=3)
        F = O.lift(d, mu, rho, a, b)
        assert abs(F @ a) < 1e-12 * np.linalg.norm(F) * np.linalg.norm(a)
        assert abs(F @ b) < 1e-12 * np.linalg.norm(F) * np.linalg.norm(b)


def test_eilers_reduces_to_einstein_and_grows():
    assert O.eilers_factor(0.0) == 1.0
    e = 1e-5
    assert (O.eilers_factor(e) - 1) / e == pytest.approx(2.5, rel=1e-4)  # Einstein: 1 + [mu] eps
    vals = [O.eilers_factor(x) for x in np.linspace(0, 0.55, 12)]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    # capped where the closure diverges (eps_p / eps_cp = 0.9)
    assert O.eilers_factor(0.63) == O.eilers_factor(0.9 * 0.64)


def test_smagorinsky_root_and_limits():
    """tau_t is the Smagorinsky relaxation time of Eq. visc_turb: with
    nu_t = c_s^2 tau_t and Sbar = Qbar/(2 rho c_s^2 (tau_* + tau_t)) it satisfies
    nu_t = C_S^2 Sbar (dx_LES = 1).  It is zero without non-equilibrium flux,
    grows with it, and equals the printed Eq. tau_t evaluated with the flux
    norm sqrt(sum Q_ab Q_ab) = Qbar / sqrt(2)."""
    Cs = 0.1
    for tau_s in (0.55, 0.8, 1.7):
        assert O.tau_turb(tau_s, 0.0, 1.0) == 0.0
        prev = 0.0
        for Q in (1e-6, 1e-4, 1e-2, 1.0):
            rho = 1.02
            t = O.tau_turb(tau_s, Q, rho)
            assert t > prev
            prev = t
            Sbar = Q / (2 * rho * CS2 * (tau_s + t))
            assert CS2 * t == pytest.approx(Cs * Cs * Sbar, rel=1e-10)
            q_h = Q / math.sqrt(2)
            printed = 0.5 * (math.sqrt(tau_s ** 2 + 2 * math.sqrt(2) * Cs * Cs * q_h / (rho * CS2 ** 2)) - tau_s)
            assert t == pytest.approx(printed, rel=1e-12)


def test_tau_e_at_equilibrium_and_with_flux():
    P = O.make_params((4, 4, 4), (1, 1, 1), tau=0.7, eilers=1, smagorinsky=1)
    u = np.array([0.01, -0.02, 0.005])
    feq = O.equilibrium(1.01, u, 0.8)
    tau_star = 0.5 + (0.7 - 0.5) * O.eilers_factor(0.2)
    assert O.tau_e(P, feq, 1.01, u, 0.8) == pytest.approx(tau_star, rel=1e-14)
    # a shear perturbation of the populations raises tau_e
    f = feq.copy()
    f += 1e-4 * C[:, 0] * C[:, 1] * W
    assert O.tau_e(P, f, 1.01, u, 0.8) > tau_star
    P0 = O.make_params((4, 4, 4), (1, 1, 1), tau=0.7)
    assert O.tau_e(P0, f, 1.01, u, 0.8) == 0.7


def test_momentum_conserved_with_all_closures():
    """Lift reactions are distributed like the added mass, and the per-cell
    relaxation time keeps the Guo momentum balance: with the pressure force
    off and f_b balancing gravity the total momentum stays constant."""
    rng = np.random.default_rng(31)
    n = (8, 8, 8)
    npart = 20
    x = rng.uniform(0, 8, size=(npart, 3))
    d = np.full(npart, 0.9)
    rho_p = np.full(npart, 2.5)
    g = np.array([0.0, 0.0, -4e-3])
    V = math.pi / 6 * d ** 3
    f_b = -((rho_p - 1.0) * V).sum() * g / (np.prod(n) - V.sum())
    P = O.make_params(n, (1, 1, 1), tau=0.7, g=g, f_b=f_b, n_int=2, n_dem=3, pressure=0, h_c=0.9, T_c=1.0,
                      e_n=0.9, lift=1, eilers=1, smagorinsky=1)
    dom = O.Domain(P, x=x, u=0.01 * rng.standard_normal((npart, 3)), d=d, rho_p=rho_p)

    def total():
        rho, j = O.moments(P, dom.f)
        m = rho_p * V
        return j.sum(1) + (m[:, None] * dom.u[:npart]).sum(0)

    t0 = total()
    dom.step(4)
    np.testing.assert_allclose(total(), t0, atol=1e-14)
    rho, _ = O.moments(P, dom.f)
    assert rho.sum() == pytest.approx(np.prod(n), rel=1e-14)
