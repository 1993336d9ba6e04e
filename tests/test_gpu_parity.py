"""GPU parity: every hot-path row of the CUDA library (through the C ABI)
against the FP64 CPU oracle on the same seeded inputs.

Tolerances: FP64 paths 1e-12 relative to the magnitude of the compared
quantity (CUDA's log/sqrt/pow/cbrt and FMA contraction differ from glibc and
the oracle's uncontracted arithmetic in the last bits); integer / index work
(the linked-cell sort) bit-exact.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1711_00336_gb300 import workloads

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _dps():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00336_gb300 import build, dps
    build.build()
    return dps


def _perm():
    """index map: library plane k holds the oracle's direction perm[k]"""
    from paper_1711_00336_gb300 import dps
    cl, _ = dps.lattice()
    co, _, _ = O.lattice()
    return np.array([next(q for q in range(19) if (co[q] == cl[k]).all()) for k in range(19)])


def close(a, b, rtol=RTOL, what="", floor=0.0):
    """max |a-b| relative to max |b|; `floor` bounds the scale from below for
    quantities that are small next to the populations they derive from (a
    lattice velocity of 1e-5 carries the round-off of O(1) populations)."""
    a, b = np.asarray(a), np.asarray(b)
    scale = max(np.abs(b).max(), floor, 1e-300)
    err = np.abs(a - b).max() / scale
    if os.environ.get("DPS_PRINT_ERR"):
        print(f"[parity] {what}: {err:.3e}")
    assert err <= rtol, f"{what}: max error {err:.3e} (relative to {scale:.3e})"


BOXES = [((8, 8, 8), (1, 1, 1)), ((13, 7, 9), (1, 1, 0)), ((6, 9, 5), (0, 0, 0)), ((3, 4, 17), (1, 0, 1))]


# ---------------------------------------------------------------------------
# S7 collide-stream (both AA parities, walls, ragged boxes)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,per", BOXES)
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_collide_stream_fp64(n, per, steps):
    dps = _dps()
    perm = _perm()
    _, w_lib = dps.lattice()
    nc = n[0] * n[1] * n[2]
    _, w_orc, _ = O.lattice()
    f0 = workloads.random_pdfs(w_orc, nc, seed=steps + nc)
    eps, fpf = workloads.random_fields(nc, seed=7 + nc)
    dom = dps.Domain(n, per, 0.62, "f64")
    dom.write_pdfs(f0[perm])
    dom.write_fields(eps_f=eps, f_pf=fpf)
    dom.collide_stream(steps)
    got = dom.read_pdfs()
    P = O.make_params(n, per, 0.62)
    ref = f0
    for _ in range(steps):
        ref = O.collide_stream(P, ref, eps, fpf)
    close(got, ref[perm], what="pdfs")
    # moments through read_fields at the new time
    fl = dom.read_fields(("rho", "ubar", "u_f", "p", "f_ext"))
    rho, j = O.moments(P, ref)
    close(fl["rho"], rho, what="rho")
    close(fl["ubar"], (j + 0.5 * fpf) / rho, what="ubar")
    close(fl["u_f"], (j + 0.5 * fpf) / rho / eps, what="u_f")
    close(fl["p"], rho / 3 / eps, what="p")
    close(fl["f_ext"], fpf, what="f_ext")
    dom.close()


def test_collide_stream_rest_state_is_exact():
    dps = _dps()
    dom = dps.Domain((7, 5, 6), (1, 0, 1), 0.9, "f64")
    _, w = dps.lattice()
    dom.collide_stream(5)
    f = dom.read_pdfs()
    # preserved to round-off (rho = sum of the weights is 1 within an ulp)
    np.testing.assert_allclose(f, np.tile(w[:, None], (1, f.shape[1])), rtol=0, atol=2e-16)
    dom.close()


# ---------------------------------------------------------------------------
# S1 linked-cell sort: bit-exact against the oracle's counting sort
# ---------------------------------------------------------------------------
def _face_particles(n, per, count, seed):
    pr = workloads.random_particles(n, per, count, seed)
    x = pr["x"]
    k = min(20, count // 4)
    x[:k] = np.floor(x[:k])  # exactly on cell faces
    for a in range(3):
        if not per[a]:  # a wall axis admits faces strictly inside the box
            x[:k, a] = np.where(x[:k, a] < 1.0, 1.0, x[:k, a])
    for a in range(3):
        if per[a]:
            x[k + a, a] = 0.0
    pr["x"] = x
    return pr


@pytest.mark.parametrize("n,per", BOXES[:3] + [((40, 33, 29), (1, 1, 0))])
def test_cell_sort_bit_exact(n, per):
    dps = _dps()
    count = 300 if n[0] > 10 else 60
    pr = _face_particles(n, per, count, seed=11)
    dom = dps.Domain(n, per, 0.7, "f64", max_particles=count)
    dom.add_particles(pr["x"], pr["d"], pr["rho_p"])
    dom.set_closure(n_int=1, n_dem=1)
    dom.prepare()
    cs, order = dom.read_cell_list()
    P = O.make_params(n, per, 0.7)
    cs_o, order_o, _ = O.cell_list(P, pr["x"], 1)
    assert np.array_equal(cs, cs_o)
    assert np.array_equal(order, order_o)
    dom.close()


def test_op_cell_sort_device_buffers():
    dps = _dps()
    import torch
    n, per = (17, 11, 9), (1, 0, 1)
    pr = _face_particles(n, per, 500, seed=5)
    x = torch.tensor(pr["x"], dtype=torch.float64, device="cuda")
    ids = torch.arange(500, dtype=torch.int32, device="cuda")
    cs, order = dps.op_cell_sort(n, per, x, ids)
    torch.cuda.synchronize()
    P = O.make_params(n, per, 0.7)
    cs_o, order_o, _ = O.cell_list(P, pr["x"], 1)
    assert np.array_equal(cs.cpu().numpy(), cs_o)
    assert np.array_equal(order.cpu().numpy(), order_o)
    # empty input: all-zero offsets
    cs0, _ = dps.op_cell_sort(n, per, x[:0], ids[:0])
    assert int(cs0.abs().sum()) == 0


# ---------------------------------------------------------------------------
# S2 eps_f
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,per", BOXES[:3])
def test_volume_fraction(n, per):
    dps = _dps()
    pr = workloads.random_particles(n, per, 50, seed=2)
    dom = dps.Domain(n, per, 0.7, "f64", max_particles=50)
    dom.add_particles(pr["x"], pr["d"], pr["rho_p"])
    dom.set_closure(n_int=1, n_dem=1, eps_min=1e-3)
    dom.prepare()
    got = dom.read_fields(("eps_f",))["eps_f"]
    P = O.make_params(n, per, 0.7, eps_min=1e-3)
    ref, _ = O.fluid_fraction(P, pr["x"], pr["d"])
    close(1 - got, 1 - ref, what="eps_p")
    dom.close()


# ---------------------------------------------------------------------------
# full coupled steps (S1-S8 together)
# ---------------------------------------------------------------------------
def _run_pair(n, per, tau, pr, steps, g=(0, 0, -2e-3), fb=(0, 0, 0), prec="f64", **kw):
    dps = _dps()
    m = len(pr["x"])
    dom = dps.Domain(n, per, tau, prec, max_particles=max(m, 1))
    if m:
        dom.add_particles(pr["x"], pr["d"], pr["rho_p"], u=pr.get("u"), w=pr.get("w"))
    dom.set_closure(g=g, fb_mode=0, fb=fb, skin=kw.pop("skin", 0.5), **kw)
    P = O.make_params(n, per, tau, g=g, f_b=fb, **kw)
    ref = O.Domain(P, x=pr["x"], u=pr.get("u"), w=pr.get("w"), d=pr["d"], rho_p=pr["rho_p"])
    dom.step(steps)
    ref.step(steps)
    return dom, ref


KW = dict(e_n=0.9, mu_c=0.25, T_c=1.0, h_c=0.5, h_min=1e-5, C_am=0.5, lub_limiter=1, lub_cap=0.25,
          eps_min=0.05)


def _packed_particles(n, per, count, seed):
    """non-overlapping spheres (d <= 1.1) with random velocities and spins"""
    pr = workloads.random_particles(n, per, count, seed)
    pr["x"] = workloads.rsa(n, per, count, 1.1, seed, margin=0.05)
    return pr


@pytest.mark.parametrize("n_int,n_dem", [(1, 1), (2, 3), (3, 2)])
@pytest.mark.parametrize("n,per", [((12, 10, 14), (1, 1, 0)), ((9, 9, 9), (1, 1, 1)), ((10, 8, 9), (0, 0, 0))])
def test_coupled_steps_fp64(n, per, n_int, n_dem):
    pr = _packed_particles(n, per, 40, seed=n_int * 10 + n_dem)
    # contacts resolved by 10 DEM substeps
    kw = {**KW, "T_c": 10.0 / (n_int * n_dem)}
    dom, ref = _run_pair(n, per, 0.7, pr, 3, n_int=n_int, n_dem=n_dem, **kw)
    got, r = dom.read_particles(), ref.particles()
    for k, fl_ in (("x", 0.0), ("u", 1e-3), ("w", 1e-3), ("F", 1e-6)):
        close(got[k], r[k], what=k, floor=fl_)
    fl, fr = dom.read_fields(("rho", "ubar", "eps_f", "f_pf")), ref.fields()
    close(fl["rho"], fr["rho"], what="rho")
    close(fl["ubar"], fr["ubar"], what="ubar", floor=1e-3)
    close(fl["eps_f"], fr["eps_f"], what="eps_f")
    close(fl["f_pf"], ref.fpf, what="f_pf", floor=1e-6)
    dom.close()


def test_single_sphere_horizon():
    """The single settling sphere (walls at z) over 200 steps: not chaotic, so
    the FP64 trajectories stay together."""
    wl = workloads.single_sphere()
    pr = dict(x=wl["x"], d=wl["d"], rho_p=wl["rho_p"])
    dom, ref = _run_pair(wl["n"], wl["periodic"], wl["tau"], pr, 200, g=wl["g"], n_int=1, n_dem=1,
                         **{**KW, "h_c": 0.8})
    got, r = dom.read_particles(), ref.particles()
    close(got["u"], r["u"], rtol=1e-11, what="u")
    close(got["x"], r["x"], rtol=1e-12, what="x")
    fl = dom.read_fields(("ubar",))
    close(fl["ubar"], ref.fields()["ubar"], rtol=1e-11, what="ubar")
    dom.close()


def test_stats_sums():
    dps = _dps()
    n, per = (10, 9, 8), (1, 1, 1)
    pr = workloads.random_particles(n, per, 30, seed=8)
    dom, ref = _run_pair(n, per, 0.8, pr, 2, n_int=2, n_dem=2, **KW)
    s = dom.stats()
    fr = ref.fields()
    rho, j = O.moments(ref.P, ref.f)
    close(s["mass"], rho.sum(), what="mass")
    close(s["fluid_j"], j.sum(1), rtol=1e-10, what="j")
    close(s["uf_mean"], fr["u_f"].mean(1), rtol=1e-10, what="uf_mean")
    m = pr["rho_p"] * np.pi / 6 * pr["d"] ** 3
    close(s["particle_momentum"], (m[:, None] * ref.particles()["u"]).sum(0), rtol=1e-10, what="p_mom")
    assert s["n_particles"] == 30 and s["step"] == 2 and s["status"] == 0
    dom.close()


def test_no_particles_is_pure_fluid():
    _dps()
    n, per = (6, 7, 8), (1, 1, 0)
    pr = dict(x=np.zeros((0, 3)), d=np.zeros(0), rho_p=np.zeros(0))
    dom, ref = _run_pair(n, per, 0.75, pr, 4, fb=(1e-5, 0, 0), n_int=2, n_dem=1, **KW)
    close(dom.read_fields(("ubar",))["ubar"], ref.fields()["ubar"], what="ubar", floor=1e-3)
    dom.close()


def test_write_particles_roundtrip_keeps_the_run_identical():
    """Reading the particles back and writing them unchanged (the e2e path of
    an external particle code) does not change the trajectory."""
    dps = _dps()
    n, per = (10, 10, 10), (1, 1, 1)
    pr = workloads.random_particles(n, per, 25, seed=4)
    runs = []
    for roundtrip in (False, True):
        dom = dps.Domain(n, per, 0.7, "f64", max_particles=25)
        dom.add_particles(pr["x"], pr["d"], pr["rho_p"], u=pr["u"], w=pr["w"])
        dom.set_closure(g=(0, 0, -1e-3), n_int=2, n_dem=2, **KW)
        for _ in range(3):
            dom.step(1)
            if roundtrip:
                p = dom.read_particles()
                dom.write_particles(p["x"], p["u"], p["w"])
        runs.append(dom.read_particles())
        dom.close()
    for k in ("x", "u"):
        assert np.array_equal(runs[0][k], runs[1][k])


def test_bad_arguments_raise():
    dps = _dps()
    dom = dps.Domain((8, 8, 8), (1, 1, 0), 0.7, "f64", max_particles=2)
    with pytest.raises(dps.DPSError):
        dom.add_particles([[1, 1, 9.0]], [1.0], [2.5])  # outside the walls
    with pytest.raises(dps.DPSError):
        dom.add_particles([[1, 1, 1.0]] * 3, [1.0] * 3, [2.5] * 3)  # capacity
    with pytest.raises(dps.DPSError):
        dom.step(1)  # no closure yet
    with pytest.raises(dps.DPSError):
        dom.set_closure(n_int=0)
    dom.close()


@pytest.mark.parametrize("eps,d", [(0.05, 1.0), (0.12, 1.0), (0.3, 1.0), (0.35, 1.2)])
def test_dense_box_lane_groups_match_the_oracle(eps, d):
    """Dense periodic boxes give each particle 2, 4 or 8 lanes in the DEM
    substep (long neighbour lists); the FP64 result still follows the oracle
    pair by pair."""
    dps = _dps()
    L = 8
    wl = workloads.settling_box(L=L, eps=eps, d=d, seed=3)
    n = len(wl["x"])
    rng = np.random.default_rng(5)
    pr = dict(x=wl["x"], d=wl["d"], rho_p=wl["rho_p"], u=0.01 * rng.standard_normal((n, 3)),
              w=0.01 * rng.standard_normal((n, 3)))
    kw = {**KW, "h_c": d, "T_c": 1.0}
    dom, ref = _run_pair((L, L, L), (1, 1, 1), 0.7, pr, 2, n_int=2, n_dem=5, **kw)
    got, r = dom.read_particles(), ref.particles()
    for k, fl_ in (("x", 0.0), ("u", 1e-3), ("w", 1e-3), ("F", 1e-6)):
        close(got[k], r[k], what=k, floor=fl_)
    close(dom.read_fields(("ubar",))["ubar"], ref.fields()["ubar"], what="ubar", floor=1e-3)
    dom.close()


def test_full_size_wall_suspension_fp64():
    """The benchmark configuration at its full size (64^3, 5000 spheres,
    walls in z, n_int = 1, n_DEM = 10, FP64) through the same public calls the
    benchmark makes: two coupled steps against the oracle, every particle and
    every cell."""
    import bench
    wl = workloads.wall_suspension()
    kw = {k: v for k, v in bench.closure_kw(wl).items() if k not in ("g", "fb", "fb_mode", "skin")}
    pr = {"x": wl["x"], "d": wl["d"], "rho_p": wl["rho_p"]}
    dom, ref = _run_pair(wl["n"], wl["periodic"], wl["tau"], pr, 2, g=wl["g"], **kw)
    got, r = dom.read_particles(), ref.particles()
    for k, fl_ in (("x", 0.0), ("u", 1e-3), ("w", 1e-3), ("F", 1e-6)):
        close(got[k], r[k], what=k, floor=fl_)
    fl, fr = dom.read_fields(("rho", "ubar", "eps_f", "f_pf")), ref.fields()
    close(fl["rho"], fr["rho"], what="rho")
    close(fl["ubar"], fr["ubar"], what="ubar", floor=1e-3)
    close(fl["eps_f"], fr["eps_f"], what="eps_f")
    close(fl["f_pf"], ref.fpf, what="f_pf", floor=1e-6)
    dom.close()
