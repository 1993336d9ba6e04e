"""Pins of the oracle's particle physics: Table 1 drag closure, Sec. 3.1.1
contact model, Sec. 3.1.3 lubrication, the integrator, Sec. 4 correlations,
and the linked-cell neighbour search against brute force."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# --------------------------------------------------------------------------
# Table 1 drag correlation
# --------------------------------------------------------------------------
def test_stokes_limit():
    """eps_p -> 0 and Re -> 0: F_d = 3 pi d mu (u_f - u_p) (Stokes' law)."""
    assert O.cd(0.0, 0.0) == pytest.approx(1.0, abs=1e-15)
    assert O.cd(1e-12, 0.0) == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("Re,expected", [(1.0, 1.15), (100.0, 1 + 0.15 * 100 ** 0.687)])
def test_single_sphere_limit_is_schiller_naumann(Re, expected):
    # Schiller-Naumann single-sphere correction; 1.15 at Re = 1
    assert O.cd(Re, 0.0) == pytest.approx(expected, rel=1e-14)


def test_drag_grows_with_solid_fraction_and_reynolds():
    es = np.linspace(0, 0.6, 13)
    vals = [O.cd(5.0, e) * (1 - e) for e in es]  # normalised F_d / F_Stokes
    assert all(b > a for a, b in zip(vals, vals[1:]))
    assert O.cd(10.0, 0.3) > O.cd(1.0, 0.3)


def test_reynolds_number_of_paper_example():
    """Sec. 4.1: u_pT = -0.048 m/s for water/glass gives Re_T = 16.8."""
    g = GOLDEN["hindered_settling_experiment"]
    Re = O.reynolds(1.0, g["rho_f"], g["d_p"], abs(g["u_pT"]), g["mu_0"])
    assert Re == pytest.approx(g["Re_T"], rel=1e-12)


def test_richardson_zaki_kappa_branches():
    assert O.rz_kappa(0.1) == 4.65
    assert O.rz_kappa(0.5) == pytest.approx(4.35 * 0.5 ** -0.03)
    assert O.rz_kappa(16.8) == pytest.approx(4.45 * 16.8 ** -0.1)
    assert O.rz_kappa(600.0) == 2.39
    # the correlation is nearly continuous at its thresholds
    for t in GOLDEN["richardson_zaki"]["thresholds"][:2]:
        assert abs(O.rz_kappa(t - 1e-9) - O.rz_kappa(t)) < 0.1


# --------------------------------------------------------------------------
# Sec. 3.1.3 lubrication against the Jeffrey-Onishi lubrication series
# --------------------------------------------------------------------------
def _jo_squeeze(lam):
    """Jeffrey & Onishi (1984) singular coefficients of X^A_11 for radius ratio lam."""
    g1 = 2 * lam ** 2 / (1 + lam) ** 3
    g2 = lam * (1 + 7 * lam + lam ** 2) / (5 * (1 + lam) ** 3)
    g3 = (1 + 18 * lam - 29 * lam ** 2 + 18 * lam ** 3 + lam ** 4) / (42 * (1 + lam) ** 3)
    return g1, g2, g3


def _jo_shear(lam):
    """Jeffrey & Onishi (1984) log coefficient of Y^A_11."""
    return 4 * lam * (2 + lam + 2 * lam ** 2) / (15 * (1 + lam) ** 3)


@pytest.mark.parametrize("xi", [1e-4, 1e-3, 1e-2, 0.1, 0.3])
def test_lubrication_equal_spheres_matches_jeffrey_onishi(xi):
    a, mu = 0.5, 0.05
    h = xi * a
    a_sq, a_sh = O.lub_coefficients(2 * a, h, mu)  # <d> = d for equal spheres
    g1, g2, g3 = _jo_squeeze(1.0)
    L = math.log(1 / xi)
    assert a_sq / (6 * math.pi * mu * a) == pytest.approx(g1 / xi + g2 * L + g3 * xi * L, rel=1e-13)
    assert a_sh / (6 * math.pi * mu * a) == pytest.approx(_jo_shear(1.0) * L, rel=1e-13)


@pytest.mark.parametrize("lam", [0.5, 2.0])
def test_lubrication_unequal_leading_order(lam):
    """Reynolds' leading term 6 pi mu (a1 a2/(a1+a2))^2 v / h for any pair."""
    a1 = 0.5
    a2 = lam * a1
    mu = 0.05
    dmean = 2 * (2 * a1) * (2 * a2) / (2 * a1 + 2 * a2)
    for h in (1e-7, 1e-8):
        a_sq, _ = O.lub_coefficients(dmean, h, mu)
        ref = 6 * math.pi * mu * (a1 * a2 / (a1 + a2)) ** 2 / h
        assert a_sq / ref == pytest.approx(1.0, rel=1e-4)


def test_lubrication_sphere_wall_leading_order():
    """Sphere-wall (<d> = 2 d_i): F -> 6 pi mu a^2 v / h (Brenner)."""
    a, mu = 0.4, 0.02
    for h in (1e-7, 1e-8):
        a_sq, _ = O.lub_coefficients(4 * a, h, mu)
        assert a_sq / (6 * math.pi * mu * a * a / h) == pytest.approx(1.0, rel=1e-4)


# --------------------------------------------------------------------------
# Sec. 3.1.1 contact model and the integrator
# --------------------------------------------------------------------------
def _dry_params(n=(16, 16, 16), periodic=(1, 1, 1), **kw):
    base = dict(tau=0.8, drag=0, pressure=0, added_mass=0, lubrication=0, contact=1,
                n_int=1, n_dem=1, pair_search=0)
    base.update(kw)
    return O.make_params(n, periodic, **base)


@pytest.mark.parametrize("e_n", [0.9, 0.5])
def test_binary_collision_restitution_and_duration(e_n):
    """Head-on dry collision of equal spheres: the linear spring-dashpot gives
    rebound ratio e_n and contact duration T_c (Eqs. damping_to_stiffness,
    collision_time), recovered as dt_DEM -> 0."""
    T_c = 1.0
    n_dem = 400
    P = _dry_params(e_n=e_n, T_c=T_c, n_dem=n_dem)
    v0 = 0.05
    x = np.array([[7.0, 8.0, 8.0], [8.0 + 0.02, 8.0, 8.0]])  # gap 0.02 with d = 1
    dom = O.Domain(P, x=x, u=[[v0, 0, 0], [-v0, 0, 0]], d=[1.0, 1.0], rho_p=[2.5, 2.5])
    contact_steps = 0
    dt = 1.0 / n_dem
    for _ in range(4):
        for _ in range(n_dem):
            # advance one DEM substep at a time through the oracle's own loop
            Fc, Tc, Fl = dom.dem_forces(dt)
            if np.abs(Fc).sum() > 0:
                contact_steps += 1
            m = 2.5 * math.pi / 6
            dom.u[:2] += dt * Fc / m
            dom.x[:2] += dt * dom.u[:2]
    vrel = dom.u[1, 0] - dom.u[0, 0]
    assert vrel / (2 * v0) == pytest.approx(e_n, rel=1e-2)
    assert contact_steps * dt == pytest.approx(T_c, rel=1e-2)


def test_contact_constants_closed_form():
    m, e, T = 0.37, 0.88, 0.5
    k, xi = O.contact_constants(m, e, T)
    # damped oscillator: period 2 pi / sqrt(k/m - (xi/2m)^2) spans 2 T_c,
    # amplitude decays by e over one half period
    wd = math.sqrt(k / m - (xi / (2 * m)) ** 2)
    assert math.pi / wd == pytest.approx(T, rel=1e-13)
    assert math.exp(-xi / (2 * m) * T) == pytest.approx(e, rel=1e-13)


def test_sliding_sphere_reaches_five_sevenths_rolling():
    """A sphere sliding on a wall without spin ends rolling at 5/7 of its
    initial speed (angular momentum about the contact point is conserved),
    which fixes the torque sign and I = m d^2 / 10."""
    g = -1e-3
    d, rho_p = 1.0, 2.5
    m = rho_p * math.pi / 6
    T_c = 1.0
    k, _ = O.contact_constants(m, 0.5, T_c)
    z0 = 0.5 - m * abs(g) / k  # resting overlap under gravity (buoyancy off: rho_f=0)
    P = _dry_params(n=(64, 8, 8), periodic=(1, 1, 0), e_n=0.5, T_c=T_c, mu_c=0.3,
                    g=(0, 0, g), rho_f=0.0, n_dem=50)
    v0 = 0.02
    dom = O.Domain(P, x=[[2.0, 4.0, z0]], u=[[v0, 0, 0]], d=[d], rho_p=[rho_p])
    dom.step(150)
    u, w = dom.u[0], dom.w[0]
    assert u[0] == pytest.approx(5 / 7 * v0, rel=2e-3)
    assert w[1] * d / 2 == pytest.approx(u[0], rel=2e-3)  # rolling: u = omega x r


def test_free_fall_semi_implicit_euler_closed_form():
    """u_k = k dt a, x_k = x_0 + dt^2 a k(k+1)/2 for constant force."""
    g = (0.0, 0.0, -2e-4)
    P = _dry_params(n=(8, 8, 32), periodic=(1, 1, 1), g=g, n_int=2, n_dem=3, contact=0)
    dom = O.Domain(P, x=[[4.0, 4.0, 20.0]], u=[[0, 0, 0]], d=[0.8], rho_p=[2.5])
    steps = 7
    dom.step(steps)
    a = (2.5 - 1.0) / 2.5 * g[2]  # (rho_p - rho_f) V g / m
    k = steps * 2 * 3
    dt = 1.0 / 6
    assert dom.u[0, 2] == pytest.approx(k * dt * a, rel=1e-13)
    assert dom.x[0, 2] == pytest.approx(20.0 + dt * dt * a * k * (k + 1) / 2, rel=1e-13)


# --------------------------------------------------------------------------
# pair forces: Newton's third law, brute force vs linked cells
# --------------------------------------------------------------------------
def _cluster(n, L, d, rng):
    x = rng.uniform(0, L, size=(n, 3))
    u = 0.01 * rng.standard_normal((n, 3))
    w = 0.01 * rng.standard_normal((n, 3))
    return x, u, w


@pytest.mark.parametrize("search", [0, 1])
def test_pair_forces_sum_to_zero_periodic(search):
    rng = np.random.default_rng(9)
    L = 6
    x, u, w = _cluster(80, L, 1.0, rng)
    P = O.make_params((L, L, L), (1, 1, 1), tau=0.7, h_c=0.5, T_c=1.0, e_n=0.8,
                      lubrication=1, contact=1, lub_limiter=0, pair_search=search)
    dom = O.Domain(P, x=x, u=u, w=w, d=np.full(80, 1.0), rho_p=np.full(80, 2.5))
    Fc, Tc, Fl = dom.dem_forces(0.01)
    assert np.abs(Fc).max() > 0 and np.abs(Fl).max() > 0
    np.testing.assert_allclose(Fc.sum(0), 0, atol=1e-12 * np.abs(Fc).max())
    np.testing.assert_allclose(Fl.sum(0), 0, atol=1e-12 * np.abs(Fl).max())


def test_linked_cells_equal_brute_force():
    rng = np.random.default_rng(10)
    L = 9
    x, u, w = _cluster(300, L, 0.9, rng)
    d = rng.uniform(0.7, 1.1, 300)
    kw = dict(tau=0.7, h_c=0.6, T_c=1.0, e_n=0.8, lubrication=1, contact=1, lub_limiter=1,
              lub_cap=0.25)
    out = []
    for search in (0, 1):
        P = O.make_params((L, L, L), (1, 1, 0), pair_search=search, **kw)
        dom = O.Domain(P, x=x, u=u, w=w, d=d, rho_p=np.full(300, 2.5))
        out.append(dom.dem_forces(0.02))
    for a, b in zip(*out):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)


def test_cell_list_structure_and_candidate_superset():
    """Sort by the bin-major cell key: a permutation, keys non-decreasing, ids
    ascending inside a key, every lattice cell a distinct key, and every pair
    within the cut-off found in neighbouring bins (checked by brute force)."""
    rng = np.random.default_rng(11)
    n = (13, 10, 11)
    P = O.make_params(n, (1, 1, 0), tau=0.7)
    B = 3
    x = rng.uniform(0, 1, size=(400, 3)) * np.array(n)
    x[:10] = np.floor(x[:10])          # exactly on cell faces
    x[10, 0] = 0.0
    cs, order, key = O.cell_list(P, x, B)
    assert sorted(order) == list(range(400))
    ks = key[order]
    assert np.all(np.diff(ks) >= 0)
    same = np.diff(ks) == 0
    assert np.all(np.diff(order)[same] > 0)
    np.testing.assert_array_equal(np.bincount(key, minlength=np.prod(n)), np.diff(cs))
    # every cell maps to a distinct key: sort a dense cloud of cell centres
    idx = np.arange(np.prod(n))
    centres = np.stack([idx % n[0], (idx // n[0]) % n[1], idx // (n[0] * n[1])], 1) + 0.5
    _, _, kc = O.cell_list(P, centres, B)
    assert sorted(kc) == list(range(np.prod(n)))
    # bins: cells of one bin occupy one contiguous key range
    nb = [max(1, m // B) for m in n]
    bins = [np.minimum((centres[:, a] // B).astype(int), nb[a] - 1) for a in range(3)]
    bid = bins[0] + nb[0] * (bins[1] + nb[1] * bins[2])
    kb = np.empty_like(kc)
    kb[:] = kc
    for b in np.unique(bid):
        kk = np.sort(kb[bid == b])
        assert kk[-1] - kk[0] + 1 == len(kk)
    # neighbour-bin candidates contain all pairs within B (brute force)
    pb = [np.minimum(np.floor(x[:, a]).astype(int) // B, nb[a] - 1) for a in range(3)]
    for i in range(0, 400, 7):
        for j in range(400):
            if i == j:
                continue
            dx = x[j] - x[i]
            for a in (0, 1):
                dx[a] -= n[a] * np.rint(dx[a] / n[a])
            if np.linalg.norm(dx) < B:
                for a in range(3):
                    db = abs(pb[a][i] - pb[a][j])
                    if a < 2:
                        db = min(db, nb[a] - db)
                    assert db <= 1


# --------------------------------------------------------------------------
# Sec. 3.1.3 with Sec. 5: lubrication acts on approaching, non-overlapping
# pairs only; a wet sphere still rebounds from a wall
# --------------------------------------------------------------------------
def test_lubrication_off_while_overlapping_on_just_before():
    P = _dry_params(lubrication=1, contact=0, h_c=0.5, h_min=1e-5)
    rel = [[0.01, 0, 0], [-0.01, 0, 0]]
    for gap, expect_lub in ((-0.01, False), (0.0, True), (1e-7, True), (0.3, True), (0.6, False)):
        x = np.array([[7.0, 8.0, 8.0], [8.0 + gap, 8.0, 8.0]])
        dom = O.Domain(P, x=x, u=rel, d=[1.0, 1.0], rho_p=[2.5, 2.5])
        _, _, Fl = dom.dem_forces(1e-3)
        assert (np.abs(Fl).max() > 0) == expect_lub, gap
        if expect_lub:
            assert Fl[0, 0] < 0 and Fl[1, 0] > 0  # resists the approach


def _wall_drop(lubrication, h_c=0.5, steps=120):
    """A heavy sphere (d = 0.5, rho_p/rho_f = 32) thrown at the bottom wall of
    a closed 12x12x24 box through fluid at rest (tau 0.505), Sec. 5 settings
    e_n = 0.97, mu_c = 0.1, T_c = 0.5, n_int = 10, n_DEM = 50."""
    P = O.make_params((12, 12, 24), (0, 0, 0), tau=0.505, g=(0, 0, -1e-4), e_n=0.97, mu_c=0.1, T_c=0.5,
                      h_c=h_c, h_min=1e-5, C_am=0.5, n_int=10, n_dem=50, lubrication=lubrication)
    dom = O.Domain(P, x=[[6.0, 6.0, 2.0]], u=[[0, 0, -0.03]], d=[0.5], rho_p=[32.0])
    u = []
    for _ in range(steps):
        dom.step(1)
        u.append(dom.u[0, 2])
    u = np.array(u)
    k = int(np.argmax(u > 0))  # first step moving up: the rebound
    return -u[k - 1], u[k:].max()


def test_wet_sphere_rebounds_less_than_dry():
    """Sec. 5: lubrication lowers the rebound (Table 3, B4 vs B0) but a
    rebound remains; without lubrication it is close to the dry e_n."""
    u_in_dry, u_out_dry = _wall_drop(lubrication=0)
    u_in_wet, u_out_wet = _wall_drop(lubrication=1)
    e_dry, e_wet = u_out_dry / u_in_dry, u_out_wet / u_in_wet
    assert 0.85 < e_dry < 1.0
    assert 0.05 < e_wet < e_dry - 0.1
