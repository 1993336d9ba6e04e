"""Pins of the oracle's GNS lattice Boltzmann model (Sec. 3.2.2: Eqs.
LBM_Equation, LBM_EQ, Forcing, MacVel; Sec. 3.2.3 lattice gradient)."""
import numpy as np
import pytest

import oracle as O

C, W, OPP = O.lattice()
CS2 = 1.0 / 3.0


def test_lattice_isotropy():
    assert W.sum() == pytest.approx(1.0, abs=1e-16)
    np.testing.assert_allclose((W[:, None] * C).sum(0), 0, atol=1e-16)
    M2 = np.einsum("q,qa,qb->ab", W, C, C)
    np.testing.assert_allclose(M2, CS2 * np.eye(3), atol=1e-16)
    M4 = np.einsum("q,qa,qb,qc,qd->abcd", W, C, C, C, C)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(M4, iso, atol=1e-16)
    for q in range(19):
        np.testing.assert_array_equal(C[OPP[q]], -C[q])


@pytest.mark.parametrize("eps", [1.0, 0.55])
def test_equilibrium_moments(eps):
    """rho, rho*ubar and rho c_s^2 I + rho ubar ubar / eps (porous equilibrium)."""
    rho, u = 1.03, np.array([0.02, -0.035, 0.011])
    feq = O.equilibrium(rho, u, eps)
    assert feq.sum() == pytest.approx(rho, rel=1e-15)
    np.testing.assert_allclose(C.T @ feq, rho * u, rtol=1e-13, atol=1e-17)
    Pi = np.einsum("q,qa,qb->ab", feq, C, C)
    np.testing.assert_allclose(Pi, rho * CS2 * np.eye(3) + rho * np.outer(u, u) / eps,
                               rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("eps", [1.0, 0.6])
def test_forcing_moments(eps):
    """Guo forcing: zero mass, (1-1/2tau) F momentum, (1-1/2tau)(uF+Fu)/eps flux."""
    tau = 0.77
    u = np.array([0.01, 0.02, -0.03])
    F = np.array([1e-3, -2e-3, 5e-4])
    Fq = O.forcing(tau, u, eps, F)
    k = 1 - 1 / (2 * tau)
    assert abs(Fq.sum()) < 1e-18
    np.testing.assert_allclose(C.T @ Fq, k * F, rtol=1e-13)
    Pi = np.einsum("q,qa,qb->ab", Fq, C, C)
    np.testing.assert_allclose(Pi, k * (np.outer(u, F) + np.outer(F, u)) / eps, rtol=1e-12,
                               atol=1e-19)


def _random_state(P, rng, amp=1e-2):
    nc = O.ncell(P)
    f = np.tile(W[:, None], (1, nc)) * (1 + amp * rng.standard_normal((19, nc)))
    eps = rng.uniform(0.6, 1.0, nc)
    fext = 1e-4 * rng.standard_normal((3, nc))
    return f, eps, fext


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 1, 0), (0, 0, 0)])
def test_collide_stream_mass_and_momentum(periodic):
    rng = np.random.default_rng(5)
    P = O.make_params((6, 5, 7), periodic, tau=0.65)
    f, eps, fext = _random_state(P, rng)
    fn = O.collide_stream(P, f, eps, fext)
    # mass: Guo forcing carries no mass, bounce-back conserves it
    assert fn.sum() == pytest.approx(f.sum(), rel=1e-14)
    if all(periodic):
        # momentum: each cell gains exactly f_ext (streaming only moves it)
        np.testing.assert_allclose((fn.T @ C).sum(0), (f.T @ C).sum(0) + fext.sum(1),
                                   rtol=0, atol=1e-14)


def test_rest_state_is_stationary():
    rng = np.random.default_rng(6)
    P = O.make_params((5, 4, 6), (1, 0, 0), tau=0.9)
    nc = O.ncell(P)
    f = np.tile(W[:, None], (1, nc)) * 1.0
    eps = rng.uniform(0.5, 1.0, nc)
    fn = O.collide_stream(P, f, eps, np.zeros((3, nc)))
    np.testing.assert_allclose(fn, f, rtol=0, atol=1e-16)


def test_streaming_moves_populations_along_their_velocity():
    """With tau=1 and a zero-velocity equilibrium the collision output is
    w_q rho; a marked population must arrive at x + c_q (periodic)."""
    P = O.make_params((4, 4, 4), (1, 1, 1), tau=1.0)
    nc = O.ncell(P)
    f = np.tile(W[:, None], (1, nc)).copy()
    eps = np.ones(nc)
    fn0 = O.collide_stream(P, f, eps, np.zeros((3, nc)))
    # perturb only the density of one cell: the change after one step is the
    # equilibrium of that cell streamed to its 19 neighbours
    c0 = 1 + 4 * (2 + 4 * 3)
    f2 = f.copy()
    f2[:, c0] *= 1.5
    fn = O.collide_stream(P, f2, eps, np.zeros((3, nc)))
    diff = fn - fn0
    for q in range(19):
        x, y, z = 1 + C[q][0], 2 + C[q][1], 3 + C[q][2]
        dst = (x % 4) + 4 * ((y % 4) + 4 * (z % 4))
        assert diff[q, dst] == pytest.approx(0.5 * W[q], rel=1e-13)
        assert np.count_nonzero(np.abs(diff[q]) > 1e-15) == 1


def _poiseuille(tau, eps, H=16, steps=None):
    """Body-force-driven channel between walls at z=0 and z=H (periodic x, y)."""
    P = O.make_params((1, 1, H), (1, 1, 0), tau=tau)
    nu = (tau - 0.5) * CS2
    g = 1e-6
    nc = H
    f = np.tile(W[:, None], (1, nc)).copy()
    epsf = np.full(nc, eps)
    fext = np.zeros((3, nc))
    fext[0] = eps * g  # f_ext = eps_f f_b
    steps = steps or int(12 * H * H / nu)
    for _ in range(steps):
        f = O.collide_stream(P, f, epsf, fext)
    rho, j = O.moments(P, f)
    ubar = (j[0] + 0.5 * fext[0]) / rho
    z = np.arange(H) + 0.5
    exact = eps * g / (2 * nu) * z * (H - z)  # ubar = eps * u_Poiseuille(f_b)
    return ubar, exact


def test_poiseuille_magic_tau_exact():
    """BGK + halfway bounce-back + Guo forcing reproduces the parabola to
    round-off at tau = 1/2 + sqrt(3/16)."""
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    ubar, exact = _poiseuille(tau, 1.0)
    np.testing.assert_allclose(ubar, exact, rtol=1e-9)


def test_poiseuille_porous_uniform_eps():
    """Uniform eps_f: the GNS equations give ubar = eps * Poiseuille(f_b)."""
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    ubar, exact = _poiseuille(tau, 0.7)
    np.testing.assert_allclose(ubar, exact, rtol=1e-9)


def test_poiseuille_tau065_close():
    ubar, exact = _poiseuille(0.65, 1.0)
    assert np.abs(ubar - exact).max() / exact.max() < 2e-2


def test_lattice_gradient_sinusoid_periodic():
    """grad sin(kx) on the D3Q19 stencil is sin(k) cos(kx) exactly."""
    L = 12
    P = O.make_params((L, 5, 4), (1, 1, 1), tau=0.8)
    idx = np.arange(O.ncell(P))
    ix = idx % L
    k = 2 * np.pi / L
    for axis_field in range(1):
        phi = np.sin(k * ix)
        g = O.lattice_gradient(P, phi)
        np.testing.assert_allclose(g[0], np.sin(k) * np.cos(k * ix), atol=1e-14)
        np.testing.assert_allclose(g[1:], 0, atol=1e-14)


def test_lattice_gradient_linear_interior_and_walls():
    n = (6, 7, 8)
    P = O.make_params(n, (0, 0, 0), tau=0.8)
    idx = np.arange(O.ncell(P))
    ix, iy, iz = idx % 6, (idx // 6) % 7, idx // 42
    a = np.array([0.3, -0.7, 1.1])
    phi = a[0] * ix + a[1] * iy + a[2] * iz
    g = O.lattice_gradient(P, phi)
    inner = (ix > 0) & (ix < 5) & (iy > 0) & (iy < 6) & (iz > 0) & (iz < 7)
    for d in range(3):
        np.testing.assert_allclose(g[d][inner], a[d], rtol=1e-13)
    # a neighbour beyond the wall is mirrored into the box: the normal
    # gradient at the wall is the one-sided half, tangential ones stay exact
    wall = (iz == 0) & (ix > 0) & (ix < 5) & (iy > 0) & (iy < 6)
    np.testing.assert_allclose(g[2][wall], a[2] / 2, rtol=1e-13)
    np.testing.assert_allclose(g[0][wall], a[0], rtol=1e-13)
