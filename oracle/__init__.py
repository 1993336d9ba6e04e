"""FP64 CPU oracle of the coupled LBM-DEM discrete particle step.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow checker that the
CUDA library is compared against; only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` import it.  It shares no code with the
CUDA library (``paper_1711_00336_gb300``) and never imports it.

Parity status of the oracle functions (what pins each one is listed in the
tests under ``tests/test_oracle_*.py``):
  - Roma kernel, distribution, interpolation, volume fraction: pinned
    (moment identities, V/8 self-interpolation, volume conservation);
  - equilibrium / Guo forcing / collide-stream: pinned (moment identities,
    Poiseuille closed form, mass and momentum balance);
  - lattice gradient: pinned (exact on linear and sinusoidal fields);
  - drag correlation: pinned at its limits only (Stokes, Schiller-Naumann,
    the Reynolds number of the paper's Sec. 4 example);
  - lubrication: pinned (Jeffrey-Onishi lubrication series, sphere-wall limit);
  - contact + integrator: pinned (dry restitution / contact time, 5/7 rolling,
    free fall closed form);
  - full coupled step: pinned by global momentum balance and the single-sphere
    slip identity; the hindered-settling trend is a loose physics check.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("periodic", ctypes.c_int * 3),
        ("tau", ctypes.c_double),
        ("rho_f", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("f_b", ctypes.c_double * 3),
        ("e_n", ctypes.c_double),
        ("mu_c", ctypes.c_double),
        ("T_c", ctypes.c_double),
        ("h_c", ctypes.c_double),
        ("h_min", ctypes.c_double),
        ("C_am", ctypes.c_double),
        ("n_int", ctypes.c_int),
        ("n_dem", ctypes.c_int),
        ("drag", ctypes.c_int),
        ("pressure", ctypes.c_int),
        ("added_mass", ctypes.c_int),
        ("lubrication", ctypes.c_int),
        ("contact", ctypes.c_int),
        ("lub_limiter", ctypes.c_int),
        ("lub_cap", ctypes.c_double),
        ("eps_min", ctypes.c_double),
        ("pair_search", ctypes.c_int),
        ("lift", ctypes.c_int),
        ("eilers", ctypes.c_int),
        ("smagorinsky", ctypes.c_int),
    ]


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


class State(ctypes.Structure):
    _fields_ = [
        ("f", _DP), ("eps_f", _DP), ("fpf", _DP), ("u_prev", _DP),
        ("have_u_prev", ctypes.c_int),
        ("np", ctypes.c_long),
        ("x", _DP), ("u", _DP), ("w", _DP), ("d", _DP), ("rho_p", _DP),
        ("u_sub", _DP), ("have_u_sub", ctypes.c_int),
        ("F_hyd", _DP), ("F_c", _DP), ("T_c", _DP), ("F_lub", _DP),
        ("n_eps_clamp", ctypes.c_long), ("n_lub_limited", ctypes.c_long),
        ("n_coincident", ctypes.c_long), ("step", ctypes.c_long),
    ]


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_phi.restype = ctypes.c_double
        L.orc_phi.argtypes = [ctypes.c_double]
        L.orc_cd.restype = ctypes.c_double
        L.orc_cd.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_reynolds.restype = ctypes.c_double
        L.orc_reynolds.argtypes = [ctypes.c_double] * 5
        L.orc_rz_kappa.restype = ctypes.c_double
        L.orc_eilers_factor.restype = ctypes.c_double
        L.orc_eilers_factor.argtypes = [ctypes.c_double]
        L.orc_tau_turb.restype = ctypes.c_double
        L.orc_tau_turb.argtypes = [ctypes.c_double] * 3
        L.orc_tau_e.restype = ctypes.c_double
        L.orc_rz_kappa.argtypes = [ctypes.c_double]
        L.orc_fluid_fraction.restype = ctypes.c_long
        L.orc_step.restype = ctypes.c_int
        _lib = L
    return _lib


def ptr(a):
    """ctypes pointer to the data of a C-contiguous float64 / int32 array."""
    if a.dtype == np.float64:
        return a.ctypes.data_as(_DP)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_IP)
    raise TypeError(a.dtype)


def make_params(n, periodic, tau, g=(0.0, 0.0, 0.0), f_b=(0.0, 0.0, 0.0), rho_f=1.0,
                e_n=0.9, mu_c=0.25, T_c=1.0, h_c=1.0, h_min=1e-5, C_am=0.5, n_int=1,
                n_dem=1, drag=1, pressure=1, added_mass=1, lubrication=1, contact=1,
                lub_limiter=1, lub_cap=0.25, eps_min=0.05, pair_search=1, lift=0, eilers=0, smagorinsky=0):
    P = Params()
    P.n[:] = [int(v) for v in n]
    P.periodic[:] = [int(bool(v)) for v in periodic]
    P.tau, P.rho_f = tau, rho_f
    P.g[:] = list(g)
    P.f_b[:] = list(f_b)
    P.e_n, P.mu_c, P.T_c, P.h_c, P.h_min, P.C_am = e_n, mu_c, T_c, h_c, h_min, C_am
    P.n_int, P.n_dem = n_int, n_dem
    P.drag, P.pressure, P.added_mass = drag, pressure, added_mass
    P.lubrication, P.contact = lubrication, contact
    P.lub_limiter, P.lub_cap, P.eps_min, P.pair_search = lub_limiter, lub_cap, eps_min, pair_search
    P.lift, P.eilers, P.smagorinsky = lift, eilers, smagorinsky
    return P


def lattice():
    c = (ctypes.c_int * 3 * 19)()
    w = (ctypes.c_double * 19)()
    opp = (ctypes.c_int * 19)()
    lib().orc_lattice(c, w, opp)
    return (np.array([[c[q][a] for a in range(3)] for q in range(19)]),
            np.array(list(w)), np.array(list(opp)))


def phi(r):
    return lib().orc_phi(float(r))


def weights_1d(xp, L, periodic):
    idx = (ctypes.c_int * 3)()
    wt = (ctypes.c_double * 3)()
    lib().orc_weights_1d(ctypes.c_double(xp), ctypes.c_int(L), ctypes.c_int(int(periodic)), idx, wt)
    return np.array(list(idx)), np.array(list(wt))


def ncell(P):
    return P.n[0] * P.n[1] * P.n[2]


def solid_fraction(P, x, d):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, np.float64)
    out = np.zeros(ncell(P))
    lib().orc_solid_fraction(ctypes.byref(P), ctypes.c_long(len(d)), ptr(x), ptr(d), ptr(out))
    return out


def fluid_fraction(P, x, d):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, np.float64)
    out = np.zeros(ncell(P))
    n = lib().orc_fluid_fraction(ctypes.byref(P), ctypes.c_long(len(d)), ptr(x), ptr(d), ptr(out))
    return out, n


def distribute(P, x, F, scale=1.0):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    F = np.ascontiguousarray(F, np.float64).reshape(-1, 3)
    out = np.zeros(3 * ncell(P))
    lib().orc_distribute(ctypes.byref(P), ctypes.c_long(len(x)), ptr(x), ptr(F),
                         ctypes.c_double(scale), ptr(out))
    return out.reshape(3, -1)


def interpolate(P, field, xp):
    field = np.ascontiguousarray(field, np.float64)
    ncomp = field.size // ncell(P)
    out = np.zeros(ncomp)
    xp = np.ascontiguousarray(xp, np.float64)
    lib().orc_interpolate(ctypes.byref(P), ptr(field.ravel()), ctypes.c_int(ncomp), ptr(xp), ptr(out))
    return out


def equilibrium(rho, u, eps):
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(19)
    lib().orc_equilibrium(ctypes.c_double(rho), ptr(u), ctypes.c_double(eps), ptr(out))
    return out


def forcing(tau, u, eps, F):
    u = np.ascontiguousarray(u, np.float64)
    F = np.ascontiguousarray(F, np.float64)
    out = np.zeros(19)
    lib().orc_forcing(ctypes.c_double(tau), ptr(u), ctypes.c_double(eps), ptr(F), ptr(out))
    return out


def moments(P, f):
    f = np.ascontiguousarray(f, np.float64)
    rho = np.zeros(ncell(P))
    j = np.zeros(3 * ncell(P))
    lib().orc_moments(ctypes.byref(P), ptr(f.ravel()), ptr(rho), ptr(j))
    return rho, j.reshape(3, -1)


def collide_stream(P, f, eps, fext):
    f = np.ascontiguousarray(f, np.float64).ravel()
    eps = np.ascontiguousarray(eps, np.float64).ravel()
    fext = np.ascontiguousarray(fext, np.float64).ravel()
    out = np.zeros_like(f)
    lib().orc_collide_stream(ctypes.byref(P), ptr(f), ptr(eps), ptr(fext), ptr(out))
    return out.reshape(19, -1)


def lattice_gradient(P, phi_field):
    phi_field = np.ascontiguousarray(phi_field, np.float64).ravel()
    out = np.zeros(3 * ncell(P))
    lib().orc_lattice_gradient(ctypes.byref(P), ptr(phi_field), ptr(out))
    return out.reshape(3, -1)


def lattice_curl(P, psi):
    psi = np.ascontiguousarray(psi, np.float64).ravel()
    out = np.zeros(3 * ncell(P))
    lib().orc_lattice_curl(ctypes.byref(P), ptr(psi), ptr(out))
    return out.reshape(3, -1)


def eilers_factor(eps_p):
    return lib().orc_eilers_factor(float(eps_p))


def tau_turb(tau_star, Qbar, rho):
    return lib().orc_tau_turb(float(tau_star), float(Qbar), float(rho))


def tau_e(P, f, rho, u, eps):
    f = np.ascontiguousarray(f, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    return lib().orc_tau_e(ctypes.byref(P), ptr(f), ctypes.c_double(rho), ptr(u), ctypes.c_double(eps))


def lift(d, mu, rho_f, du, w):
    du = np.ascontiguousarray(du, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    out = np.zeros(3)
    lib().orc_lift(ctypes.c_double(d), ctypes.c_double(mu), ctypes.c_double(rho_f), ptr(du), ptr(w), ptr(out))
    return out


def cd(Re, eps_p):
    return lib().orc_cd(float(Re), float(eps_p))


def reynolds(eps_f, rho_f, d, du, mu):
    return lib().orc_reynolds(float(eps_f), float(rho_f), float(d), float(du), float(mu))


def rz_kappa(Re_T):
    return lib().orc_rz_kappa(float(Re_T))


def contact_constants(m_ij, e_n, T_c):
    k = ctypes.c_double()
    xi = ctypes.c_double()
    lib().orc_contact_constants(ctypes.c_double(m_ij), ctypes.c_double(e_n), ctypes.c_double(T_c),
                                ctypes.byref(k), ctypes.byref(xi))
    return k.value, xi.value


def lub_coefficients(dmean, h, mu):
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib().orc_lub_coefficients(ctypes.c_double(dmean), ctypes.c_double(h), ctypes.c_double(mu),
                               ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def cell_list(P, x, B):
    """Linked-cell sort: (cell_start[ncell+1], order[np], key[np])."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    npart = len(x)
    cs = np.zeros(ncell(P) + 1, np.int32)
    order = np.zeros(max(npart, 1), np.int32)
    key = np.zeros(max(npart, 1), np.int32)
    lib().orc_cell_list(ctypes.byref(P), ctypes.c_long(npart), ptr(x), ctypes.c_int(B),
                        ptr(cs), ptr(order), ptr(key))
    return cs, order[:npart], key[:npart]


class Domain:
    """Oracle state of one box: fluid fields and particles, owned as numpy arrays."""

    def __init__(self, P, x=None, u=None, w=None, d=None, rho_p=None):
        self.P = P
        nc = ncell(P)
        x = np.zeros((0, 3)) if x is None else np.asarray(x, np.float64).reshape(-1, 3)
        npart = len(x)
        self.f = np.zeros((19, nc))
        self.eps_f = np.zeros(nc)
        self.fpf = np.zeros((3, nc))
        self.u_prev = np.zeros((3, nc))
        m = max(npart, 1)

        def vec(v):
            a = np.zeros((m, 3))
            if v is not None and npart:
                a[:npart] = np.asarray(v, np.float64).reshape(-1, 3)
            return a

        self.x = vec(x)
        self.u = vec(u)
        self.w = vec(w)
        self.d = np.ones(m)
        self.rho_p = np.ones(m)
        if npart:
            self.d[:npart] = np.broadcast_to(np.asarray(d, np.float64), (npart,))
            self.rho_p[:npart] = np.broadcast_to(np.asarray(rho_p, np.float64), (npart,))
        self.u_sub = np.zeros((m, 3))
        self.F_hyd = np.zeros((m, 3))
        self.F_c = np.zeros((m, 3))
        self.T_c = np.zeros((m, 3))
        self.F_lub = np.zeros((m, 3))
        S = State()
        for name in ("f", "eps_f", "fpf", "u_prev", "x", "u", "w", "d", "rho_p", "u_sub",
                     "F_hyd", "F_c", "T_c", "F_lub"):
            setattr(S, name, ptr(getattr(self, name)))
        S.np = npart
        self.S = S
        self.np = npart
        lib().orc_init(ctypes.byref(P), ctypes.byref(S))

    def step(self, n=1):
        rc = lib().orc_step(ctypes.byref(self.P), ctypes.byref(self.S), ctypes.c_long(n))
        if rc != 0:
            raise MemoryError("oracle step failed")

    def dem_forces(self, dt_dem):
        lib().orc_dem_forces(ctypes.byref(self.P), ctypes.byref(self.S), ctypes.c_double(dt_dem))
        n = self.np
        return self.F_c[:n].copy(), self.T_c[:n].copy(), self.F_lub[:n].copy()

    # views
    def particles(self):
        n = self.np
        return dict(x=self.x[:n].copy(), u=self.u[:n].copy(), w=self.w[:n].copy(),
                    F=self.F_hyd[:n].copy())

    def fields(self):
        """rho, ubar (3), u_f (3), eps_f, f_ext (3) at the current time."""
        P = self.P
        rho, j = moments(P, self.f)
        fext = self.fpf + self.eps_f[None, :] * np.asarray(list(P.f_b))[:, None]
        ubar = (j + 0.5 * fext) / rho[None, :]
        return dict(rho=rho, ubar=ubar, u_f=ubar / self.eps_f[None, :], eps_f=self.eps_f.copy(),
                    f_ext=fext)

    @property
    def counters(self):
        return dict(eps_clamp=self.S.n_eps_clamp, lub_limited=self.S.n_lub_limited,
                    coincident=self.S.n_coincident, step=self.S.step)
