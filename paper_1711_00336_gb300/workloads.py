"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke
check.  Only random numbers and geometry live here (positions, random PDF and
field perturbations, box descriptions); none of the method's arithmetic does.

Workloads (lattice units, Sec. 3.2.2):
  single_sphere   32x32x64, walls at z = 0 and 64, tau 0.65, one sphere d = 0.8,
                  rho_p/rho_f = 2.5 released at (16,16,48); gravity set from the
                  Stokes closed form for a particle Reynolds number of 0.1.
  wall_suspension 64^3, walls at z, 5000 spheres d = 1, rho_p/rho_f = 2.5, random
                  sequential insertion (non-overlapping, seed 12345).
  settling_box    triply periodic L^3, spheres of diameter d at a solid volume
                  fraction eps: random sequential insertion below 0.3, above it a
                  random subset of a jittered cubic lattice (non-overlapping);
                  tau 0.55, rho_p/rho_f 2.5, gravity for a Stokes Reynolds
                  number of 0.1; beyond the cubic lattice's limit a jittered
                  face-centred cubic subset (up to 0.74).
"""
import math

import numpy as np


def stokes_gravity(tau, d, rho_ratio, Re=0.1):
    """|g| such that the Stokes settling velocity of one sphere has Reynolds
    number Re: u_St = Re nu / d, g = 18 mu u_St / ((rho_p - rho_f) d^2)."""
    nu = (tau - 0.5) / 3.0
    u_st = Re * nu / d
    return 18.0 * nu * u_st / ((rho_ratio - 1.0) * d * d), u_st


def single_sphere():
    tau, d, rr = 0.65, 0.8, 2.5
    g, u_st = stokes_gravity(tau, d, rr)
    return dict(name="single_sphere_32x32x64", n=(32, 32, 64), periodic=(1, 1, 0), tau=tau,
                x=np.array([[16.0, 16.0, 48.0]]), d=np.array([d]), rho_p=np.array([rr]),
                g=(0.0, 0.0, -g), u_st=u_st, steps=2000)


def rsa(n, periodic, count, d, seed, margin=0.0, max_tries=200):
    """Random sequential insertion of `count` non-overlapping spheres of
    diameter d (grid-accelerated).  On wall axes centres keep d/2 + margin
    from the faces."""
    rng = np.random.default_rng(seed)
    n = np.asarray(n, float)
    lo = np.array([0.0 if p else d / 2 + margin for p in periodic])
    hi = np.array([n[a] if periodic[a] else n[a] - d / 2 - margin for a in range(3)])
    cell = d
    gdim = np.maximum((n // cell).astype(int), 1)
    grid = {}
    pts = np.zeros((count, 3))
    k = 0
    tries = 0
    while k < count:
        tries += 1
        if tries > max_tries * count:
            raise RuntimeError("random sequential insertion jammed")
        p = lo + rng.random(3) * (hi - lo)
        g = tuple((p // (n / gdim)).astype(int) % gdim)
        ok = True
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    key = ((g[0] + dx) % gdim[0], (g[1] + dy) % gdim[1], (g[2] + dz) % gdim[2])
                    for q in grid.get(key, ()):
                        v = pts[q] - p
                        for a in range(3):
                            if periodic[a]:
                                v[a] -= n[a] * round(v[a] / n[a])
                        if v @ v < d * d:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pts[k] = p
            grid.setdefault(g, []).append(k)
            k += 1
    return pts


def jittered_lattice(L, count, d, seed):
    """`count` spheres on a random subset of a cubic lattice filling a periodic
    L^3 box, each displaced by at most (a - d)/2 per axis (no overlaps).  The
    spacing a is at least 1.02 d where the sites suffice, so that lattice
    neighbours do not start in exact contact."""
    rng = np.random.default_rng(seed)
    m = int(math.floor(L / (1.02 * d)))
    if m ** 3 < count:
        m = int(math.floor(L / d))
    if m ** 3 < count:
        raise ValueError("volume fraction above the cubic-lattice limit")
    a = L / m
    sites = rng.choice(m ** 3, size=count, replace=False)
    ijk = np.stack([sites % m, (sites // m) % m, sites // (m * m)], 1).astype(float)
    jit = (a - d) / 2 * 0.999
    pts = (ijk + 0.5) * a + rng.uniform(-jit, jit, size=(count, 3))
    return np.mod(pts, L)


def fcc_lattice(L, count, d, seed):
    """`count` spheres on a random subset of a face-centred cubic lattice
    filling a periodic L^3 box (cubic cells of edge a, four sites each),
    nearest neighbours a/sqrt(2) >= 1.02 d apart where the sites suffice,
    each sphere displaced by less than half the spare gap (no overlaps):
    packings up to a solid fraction of 0.74."""
    rng = np.random.default_rng(seed)
    m = int(math.floor(L / (math.sqrt(2.0) * 1.02 * d)))
    if 4 * m ** 3 < count:
        m = int(math.floor(L / (math.sqrt(2.0) * d)))
    if 4 * m ** 3 < count:
        raise ValueError("volume fraction above the face-centred cubic limit")
    a = L / m
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    sites = rng.choice(4 * m ** 3, size=count, replace=False)
    cell, b = sites // 4, sites % 4
    ijk = np.stack([cell % m, (cell // m) % m, cell // (m * m)], 1).astype(float)
    jit = (a / math.sqrt(2.0) - d) / 2 * 0.999 / math.sqrt(3.0)
    pts = (ijk + basis[b] + 0.25) * a + rng.uniform(-jit, jit, size=(count, 3))
    return np.mod(pts, L)


def wall_suspension(seed=12345, n=(64, 64, 64), count=5000, d=1.0):
    tau, rr = 0.65, 2.5
    g, u_st = stokes_gravity(tau, d, rr)
    x = rsa(n, (1, 1, 0), count, d, seed, margin=0.05)
    return dict(name=f"wall_suspension_{n[0]}x{n[1]}x{n[2]}_N{count}", n=n, periodic=(1, 1, 0), tau=tau,
                x=x, d=np.full(count, d), rho_p=np.full(count, rr), g=(0.0, 0.0, -g), u_st=u_st, steps=5000)


def settling_count(L, eps, d):
    """number of spheres of diameter d giving solid volume fraction eps in L^3"""
    return int(round(eps * L ** 3 / (math.pi / 6 * d ** 3)))


def settling_box(L=64, eps=0.2, d=1.5, seed=1, tau=0.55, Re=0.1):
    count = settling_count(L, eps, d)
    if eps <= 0.3 and count <= 60000:
        x = rsa((L, L, L), (1, 1, 1), count, d, seed)
    elif int(math.floor(L / d)) ** 3 >= count:
        x = jittered_lattice(L, count, d, seed)
    else:
        x = fcc_lattice(L, count, d, seed)
    g, u_st = stokes_gravity(tau, d, 2.5, Re)
    return dict(name=f"settling_{L}^3_eps{eps}_d{d}", n=(L, L, L), periodic=(1, 1, 1), tau=tau, x=x,
                d=np.full(count, d), rho_p=np.full(count, 2.5), g=(0.0, 0.0, -g), u_st=u_st)


def random_pdfs(w, ncell, seed, amp=0.01):
    """f_q = w_q (1 + amp*xi) with xi standard normal, given weights w[19]."""
    rng = np.random.default_rng(seed)
    return w[:, None] * (1.0 + amp * rng.standard_normal((len(w), ncell)))


def random_fields(ncell, seed, eps_range=(0.6, 1.0), force_amp=1e-4):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(*eps_range, size=ncell)
    fpf = force_amp * rng.standard_normal((3, ncell))
    return eps, fpf


def random_particles(n, periodic, count, seed, d_range=(0.7, 1.1), speed=0.01):
    """Uniform positions (overlaps allowed), small random velocities/spins."""
    rng = np.random.default_rng(seed)
    n = np.asarray(n, float)
    lo = np.array([0.0 if p else 0.6 for p in periodic])
    hi = np.array([n[a] if periodic[a] else n[a] - 0.6 for a in range(3)])
    x = lo + rng.random((count, 3)) * (hi - lo)
    return dict(x=x, u=speed * rng.standard_normal((count, 3)), w=speed * rng.standard_normal((count, 3)),
                d=rng.uniform(*d_range, size=count), rho_p=np.full(count, 2.5))
