"""Precision forms against the FP64 oracle: PDFs stored FP32 or FP16 as
shifted populations f_q - w_q rho_0 with FP32 arithmetic; particles FP64.

Stated tolerances (velocity field, relative L2 over the box):
  FP32 form       1e-4 after 100 steps
  FP16-shifted    5e-3 after 100 steps
and the settling velocity of the single-sphere workload within 1 % of the
FP64 oracle in every form."""
import numpy as np
import pytest

import oracle as O
from paper_1711_00336_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL_FIELD = {"f32": 1e-4, "f16s": 5e-3}


def _dps():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00336_gb300 import build, dps
    build.build()
    return dps


def _perm():
    from paper_1711_00336_gb300 import dps
    cl, _ = dps.lattice()
    co, _, _ = O.lattice()
    return np.array([next(q for q in range(19) if (co[q] == cl[k]).all()) for k in range(19)])


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_collide_stream_forms(prec):
    dps = _dps()
    n, per = (16, 12, 10), (1, 1, 0)
    nc = int(np.prod(n))
    _, w, _ = O.lattice()
    # a smooth shear-wave initial state (velocity 1e-2) and a uniform force
    idx = np.arange(nc)
    iy = (idx // n[0]) % n[1]
    u = 0.01 * np.sin(2 * np.pi * iy / n[1])
    f0 = np.stack([O.equilibrium(1.0, np.array([u[c], 0.0, 0.0]), 1.0) for c in range(nc)], 1)
    eps = np.full(nc, 0.9)
    fpf = np.zeros((3, nc))
    fpf[0] = 1e-6
    dom = dps.Domain(n, per, 0.65, prec)
    dom.write_pdfs(f0[_perm()])
    dom.write_fields(eps_f=eps, f_pf=fpf)
    dom.collide_stream(100)
    got = dom.read_fields(("ubar",))["ubar"]
    P = O.make_params(n, per, 0.65)
    ref = f0
    for _ in range(100):
        ref = O.collide_stream(P, ref, eps, fpf)
    rho, j = O.moments(P, ref)
    ub = (j + 0.5 * fpf) / rho
    assert rel_l2(got, ub) < TOL_FIELD[prec]
    dom.close()


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_single_sphere_settling_velocity_forms(prec):
    """Terminal settling velocity of the single sphere within 1 % of FP64."""
    dps = _dps()
    wl = workloads.single_sphere()
    kw = dict(e_n=0.9, mu_c=0.25, T_c=1.0, h_c=0.8, h_min=1e-5, C_am=0.5, n_int=1, n_dem=1, lub_limiter=1,
              lub_cap=0.25, eps_min=0.05)
    res = {}
    for p in ("f64", prec):
        dom = dps.Domain(wl["n"], wl["periodic"], wl["tau"], p, max_particles=1)
        dom.add_particles(wl["x"], wl["d"], wl["rho_p"])
        dom.set_closure(g=wl["g"], fb_mode=0, fb=(0, 0, 0), skin=0.5, **kw)
        dom.step(600)
        res[p] = (dom.read_particles()["u"][0, 2], dom.read_fields(("u_f",))["u_f"])
        dom.close()
    assert abs(res[prec][0] - res["f64"][0]) / abs(res["f64"][0]) < 1e-2
    assert rel_l2(res[prec][1], res["f64"][1]) < 10 * TOL_FIELD[prec]


def test_f64_gpu_single_sphere_matches_oracle_terminal_velocity():
    """The FP64 GPU path and the oracle agree on the terminal velocity over
    the first 600 steps of the single-sphere workload."""
    dps = _dps()
    wl = workloads.single_sphere()
    kw = dict(e_n=0.9, mu_c=0.25, T_c=1.0, h_c=0.8, h_min=1e-5, C_am=0.5, n_int=1, n_dem=1, lub_limiter=1,
              lub_cap=0.25, eps_min=0.05)
    dom = dps.Domain(wl["n"], wl["periodic"], wl["tau"], "f64", max_particles=1)
    dom.add_particles(wl["x"], wl["d"], wl["rho_p"])
    dom.set_closure(g=wl["g"], fb_mode=0, fb=(0, 0, 0), skin=0.5, **kw)
    dom.step(600)
    u = dom.read_particles()["u"][0, 2]
    P = O.make_params(wl["n"], wl["periodic"], wl["tau"], g=wl["g"], **kw)
    ref = O.Domain(P, x=wl["x"], d=wl["d"], rho_p=wl["rho_p"])
    ref.step(600)
    assert abs(u - ref.u[0, 2]) / abs(ref.u[0, 2]) < 1e-10
    dom.close()


@pytest.mark.parametrize("prec", ["f32", "f16s"])
@pytest.mark.parametrize("n,per", [((8, 8, 8), (1, 1, 1)), ((13, 7, 9), (1, 1, 0)), ((6, 9, 5), (0, 0, 0)),
                                   ((3, 4, 17), (1, 0, 1)), ((40, 5, 6), (1, 0, 1)), ((37, 6, 5), (0, 1, 1))])
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_collide_stream_forms_every_population_lands(prec, n, per, steps):
    """One to three collide-stream steps of the low-precision forms (both AA
    parities, the odd one warp-cooperative) on ragged boxes with walls and
    periodic faces: every population agrees with the FP64 oracle to the
    storage precision (a misplaced population would be off by ~1e-3)."""
    dps = _dps()
    perm = _perm()
    nc = int(np.prod(n))
    _, w, _ = O.lattice()
    from paper_1711_00336_gb300 import workloads
    f0 = workloads.random_pdfs(w, nc, seed=steps + nc, amp=0.02)
    eps, fpf = workloads.random_fields(nc, seed=3 + nc)
    dom = dps.Domain(n, per, 0.62, prec)
    dom.write_pdfs(f0[perm])
    dom.write_fields(eps_f=eps, f_pf=fpf)
    dom.collide_stream(steps)
    got = dom.read_pdfs()
    P = O.make_params(n, per, 0.62)
    ref = f0
    for _ in range(steps):
        ref = O.collide_stream(P, ref, eps, fpf)
    tol = {"f32": 2e-7, "f16s": 2e-4}[prec]
    assert np.abs(got - ref[perm]).max() < tol
    dom.close()


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_mixed_dem_pairs_near_contact_at_large_coordinates(prec):
    """The low-precision forms take the separation of a pair near contact
    (gap below 1e-3 dx, or overlapping) from the FP64 positions: sphere pairs
    around x = 200, where the float copies of the positions are ~1.5e-5
    coarse, with gaps from an overlap of 2e-3 to 1.5e-3, approaching one
    another, follow the FP64 oracle through contact and lubrication
    (hydrodynamic forces off) to 1e-5 of the largest velocity; the separation
    from the float copies alone would be off by several per cent for these
    gaps (4e-4 of the largest velocity).  Two pairs away from contact (gaps
    0.05 and 0.3, separation from the float copies) sit near x = 20, where
    the copies are fine enough for that bound."""
    dps = _dps()
    n, per = (224, 12, 12), (1, 1, 1)
    gaps = [-2e-3, -5e-4, 0.0, 2e-4, 8e-4, 1.5e-3, 0.05, 0.3]
    th = 0.3
    x, u = [], []
    for k, gp in enumerate(gaps):
        y, z = 1.5 + 3.0 * (k % 4), 3.0 + 6.0 * (k // 4)
        x0 = (200.37 if abs(gp) < 2e-3 else 20.37) + 0.113 * k
        x.append([x0, y, z])
        x.append([x0 + (1.0 + gp) * np.cos(th), y + (1.0 + gp) * np.sin(th), z])
        u.append([1e-3, 0.0, 2e-4])
        u.append([-1e-3, 1e-4, 0.0])
    x, u = np.array(x), np.array(u)
    w = np.random.default_rng(5).normal(0.0, 1e-3, x.shape)
    npart = len(x)
    kw = dict(e_n=0.9, mu_c=0.25, T_c=1.0, h_c=1.0, h_min=1e-5, C_am=0.5, n_int=1, n_dem=10, drag=0, pressure=0,
              added_mass=0, lub_limiter=1, lub_cap=0.25, eps_min=0.05)
    dom = dps.Domain(n, per, 0.6, prec, max_particles=npart)
    dom.add_particles(x, np.ones(npart), np.full(npart, 2.5), u=u, w=w)
    dom.set_closure(g=(0.0, 0.0, 0.0), fb_mode=0, skin=0.5, **kw)
    dom.step(2)
    got = dom.read_particles()
    dom.close()
    P = O.make_params(n, per, 0.6, **kw)
    ref = O.Domain(P, x=x, u=u, w=w, d=np.ones(npart), rho_p=np.full(npart, 2.5))
    ref.step(2)
    r = ref.particles()
    assert np.abs(got["u"] - r["u"]).max() < 1e-5 * np.abs(r["u"]).max()
    assert np.abs(got["w"] - r["w"]).max() < 1e-5 * np.abs(r["w"]).max()
    # the pairs in contact or within lubrication range changed velocity
    assert np.abs(r["u"] - u)[:12].max() > 1e-4
