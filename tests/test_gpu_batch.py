"""Batching and serving forms: many uneven boxes advanced by one launch per
phase must give every box exactly the result it gets alone (its kernels
touch only its own data, in the same order), for any launch shape; the
serving loop must reproduce a request's result whether it ran alone or among
others, and admit / retire boxes as memory and convergence dictate."""
import time

import numpy as np
import pytest

import oracle as O
from paper_1711_00336_gb300 import workloads

pytestmark = pytest.mark.gpu


def _dps():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00336_gb300 import build, dps
    build.build()
    return dps


KW = dict(e_n=0.88, mu_c=0.25, T_c=0.5, h_min=1e-5, C_am=0.5, n_int=2, n_dem=5, lub_limiter=1, lub_cap=0.25,
          eps_min=0.05, skin=0.5, fb_mode=1)


def _boxes():
    """three uneven periodic boxes with different d and volume fraction"""
    out = []
    for L, eps, d, seed in ((14, 0.1, 0.8, 1), (19, 0.25, 1.2, 2), (11, 0.05, 1.5, 3)):
        wl = workloads.settling_box(L=L, eps=eps, d=d, seed=seed)
        out.append(wl)
    return out


def _closure(dps, wl):
    return dps.closure(g=wl["g"], h_c=wl["d"][0], **KW)


def _alone(dps, wl, prec, steps):
    dom = dps.Domain(wl["n"], wl["periodic"], wl["tau"], prec, max_particles=len(wl["x"]))
    dom.add_particles(wl["x"], wl["d"], wl["rho_p"])
    dom.set_closure(_closure(dps, wl))
    dom.step(steps)
    r = dom.read_particles()
    f = dom.read_fields(("ubar",))["ubar"]
    dom.close()
    return r, f


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_equals_each_box_alone(prec):
    dps = _dps()
    wls = _boxes()
    steps = 6
    B = dps.Batch(prec)
    ids = []
    for wl in wls:
        b = B.add_box(wl["n"], wl["periodic"], wl["tau"], len(wl["x"]))
        B.add_particles(b, wl["x"], wl["d"], wl["rho_p"])
        B.set_closure(b, _closure(dps, wl))
        ids.append(b)
    B.step(steps)
    for b, wl in zip(ids, wls):
        r, f = _alone(dps, wl, prec, steps)
        got = B.read_particles(b)
        assert np.array_equal(got["x"], r["x"]) and np.array_equal(got["u"], r["u"])
        assert np.array_equal(B.read_fields(b, ("ubar",))["ubar"], f)
    B.close()


def test_launch_shape_does_not_change_results():
    dps = _dps()
    wl = _boxes()[1]
    res = []
    for cfg in ([128, 1024, 128, 256, 0], [64, 256, 64, 64, 1], [256, 4096, 256, 512, 2], [128, 2048, 32, 32, 3],
                [256, 1024, 128, 128, 4], [128, 1024, 64, 256, 5]):
        B = dps.Batch("f32")
        b = B.add_box(wl["n"], wl["periodic"], wl["tau"], len(wl["x"]))
        B.add_particles(b, wl["x"], wl["d"], wl["rho_p"])
        B.set_closure(b, _closure(dps, wl))
        B.set_tuning(cfg)
        B.step(4)
        res.append(B.read_particles(b)["u"])
        B.close()
    for r in res[1:]:
        assert np.array_equal(res[0], r)


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_vector_pair_collide_variants_give_the_same_bits(prec):
    """Collide-stream variants 6 and 7 move two adjacent cells' populations as
    two-element vectors (even nx; pairs next to a wall, and odd nx, take the
    scalar path): every PDF-derived field and particle must equal the scalar
    variant's bits, at both AA parities, in periodic and walled boxes."""
    dps = _dps()
    boxes = [((16, 12, 10), (1, 1, 1)), ((16, 10, 12), (0, 1, 1)), ((12, 14, 16), (1, 1, 0)), ((13, 8, 10), (1, 0, 1))]
    for n, per in boxes:
        pr = workloads.random_particles(n, per, 30, seed=n[0], d_range=(0.8, 1.0), speed=0.005)
        pr["x"] = workloads.rsa(n, per, 30, 1.0, n[0], margin=0.05)
        res = []
        for variant in (3, 6, 7):
            B = dps.Batch(prec)
            b = B.add_box(n, per, 0.6, 30)
            B.add_particles(b, pr["x"], pr["d"], pr["rho_p"], u=pr["u"], w=pr["w"])
            B.set_closure(b, dps.closure(g=(0, 0, -2e-3), h_c=0.5, **KW))
            B.set_tuning([128, 1024, 128, 256, variant])
            B.step(3)  # odd: the last step ran at the odd parity
            f3 = B.read_fields(b, ("rho", "ubar", "f_pf"))
            B.step(1)
            f4 = B.read_fields(b, ("rho", "ubar"))
            res.append((f3, f4, B.read_particles(b)["u"]))
            B.close()
        for f3, f4, u in res[1:]:
            for k in f3:
                assert np.array_equal(f3[k], res[0][0][k]), (n, per, k)
            for k in f4:
                assert np.array_equal(f4[k], res[0][1][k]), (n, per, k)
            assert np.array_equal(u, res[0][2])


def test_autotune_keeps_a_valid_shape_and_removal_leaves_others_untouched():
    dps = _dps()
    wls = _boxes()
    B = dps.Batch("f32")
    ids = []
    for wl in wls:
        b = B.add_box(wl["n"], wl["periodic"], wl["tau"], len(wl["x"]))
        B.add_particles(b, wl["x"], wl["d"], wl["rho_p"])
        B.set_closure(b, _closure(dps, wl))
        ids.append(b)
    ms = B.autotune(steps=2)
    assert ms > 0
    cfg = B.tuning()
    assert cfg[0] % 32 == 0 and cfg[2] % 32 == 0
    steps_done = B.stats(ids[0])["step"]  # every candidate ran a capture step and the timed steps
    assert steps_done % 3 == 0 and steps_done >= 3 * 12
    B.remove_box(ids[1])
    B.step(3)
    r, _ = _alone(dps, wls[0], "f32", steps_done + 3)
    assert np.array_equal(B.read_particles(ids[0])["x"], r["x"])
    B.close()


def test_batch_fp64_box_matches_oracle():
    dps = _dps()
    wl = workloads.settling_box(L=10, eps=0.15, d=1.0, seed=9)
    B = dps.Batch("f64")
    b = B.add_box(wl["n"], wl["periodic"], wl["tau"], len(wl["x"]))
    B.add_particles(b, wl["x"], wl["d"], wl["rho_p"])
    c = _closure(dps, wl)
    B.set_closure(b, c)
    B.step(3)
    got = B.read_particles(b)
    V = np.pi / 6 * wl["d"] ** 3
    fb = -((wl["rho_p"] - 1) * V).sum() * np.asarray(wl["g"]) / (np.prod(wl["n"]) - V.sum())
    kw = {k: v for k, v in KW.items() if k not in ("skin", "fb_mode")}
    P = O.make_params(wl["n"], wl["periodic"], wl["tau"], g=wl["g"], f_b=fb, h_c=wl["d"][0], **kw)
    ref = O.Domain(P, x=wl["x"], d=wl["d"], rho_p=wl["rho_p"])
    ref.step(3)
    r = ref.particles()
    err = np.abs(got["u"] - r["u"]).max() / max(np.abs(r["u"]).max(), 1e-3)
    assert err < 1e-12
    B.close()


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
def _request(dps, L, eps, seed, d=1.0):
    wl = workloads.settling_box(L=L, eps=eps, d=d, seed=seed)
    c = dps.closure(g=wl["g"], h_c=d, **KW)
    return wl, c


def test_serving_result_is_the_same_alone_and_in_the_mix():
    dps = _dps()
    reqs = [_request(dps, L, e, s) for L, e, s in ((16, 0.1, 1), (12, 0.2, 2), (20, 0.05, 3))]
    kw = dict(max_steps=600, window=200, rel_tol=1e-9)  # run to the cap: deterministic length
    S = dps.Server("f32", max_boxes=8, hbm_reserve_bytes=1 << 30, chunk_steps=50)
    wl, c = reqs[0]
    rid = S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], c, **kw)
    S.wait_idle(600)
    alone = S.poll(rid)
    S.close()
    assert alone["state"] == "done" and alone["steps"] == 600
    S = dps.Server("f32", max_boxes=8, hbm_reserve_bytes=1 << 30, chunk_steps=50)
    ids = []
    for k, (wl, c) in enumerate(reqs[::-1]):  # request 0 arrives last, joins a running batch
        ids.append(S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], c, **kw))
        time.sleep(0.05)
    S.wait_idle(600)
    mixed = S.poll(ids[-1])
    st = S.stats()
    S.close()
    assert mixed["state"] == "done", mixed
    assert np.array_equal(mixed["up_mean"], alone["up_mean"]), (mixed, alone)
    assert np.array_equal(mixed["u_pS"], alone["u_pS"]), (mixed, alone)
    assert st["completed"] == 3 and st["cell_updates"] > 0


def test_serving_convergence_cancel_and_admission():
    dps = _dps()
    S = dps.Server("f32", max_boxes=2, hbm_reserve_bytes=1 << 30, chunk_steps=50)
    wl, c = _request(dps, 12, 0.1, 4)
    a = S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], c, max_steps=20000,
                 window=500, rel_tol=1e-3)
    b = S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], c, max_steps=20000,
                 window=500, rel_tol=1e-3)
    cc = S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], c, max_steps=20000,
                  window=500, rel_tol=1e-3)
    S.cancel(cc)  # third request waits for a slot and is cancelled there
    # a box that can never fit in HBM fails at admission without allocating
    big = S.submit((1200, 1200, 1200), (1, 1, 1), 0.65, wl["x"][:1], wl["d"][:1], wl["rho_p"][:1], c,
                   max_steps=100, window=50, rel_tol=1e-3)
    S.wait_idle(900)
    ra, rb, rc, rbig = S.poll(a), S.poll(b), S.poll(cc), S.poll(big)
    S.close()
    assert ra["state"] == "done" and rb["state"] == "done"
    assert ra["steps"] % 500 == 0
    assert np.array_equal(ra["up_mean"], rb["up_mean"])
    assert rc["state"] == "cancelled"
    assert rbig["state"] == "failed"


def test_serving_failing_request_leaves_the_others_running():
    """A request whose particles leave their neighbour-list skin (gravity far
    too strong for its subcycle) fails alone; the request running beside it
    completes with the result it has alone."""
    dps = _dps()
    kw = dict(max_steps=300, window=100, rel_tol=1e-9)
    wl, c = _request(dps, 12, 0.1, 5)
    S = dps.Server("f32", max_boxes=4, hbm_reserve_bytes=1 << 30, chunk_steps=50)
    alone = S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], c, **kw)
    S.wait_idle(600)
    r_alone = S.poll(alone)
    S.close()
    bad_c = dps.closure(g=(0.0, 0.0, -5.0), h_c=1.0, **KW)
    S = dps.Server("f32", max_boxes=4, hbm_reserve_bytes=1 << 30, chunk_steps=50)
    good = S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], c, **kw)
    bad = S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], bad_c, **kw)
    S.wait_idle(600)
    rg, rb = S.poll(good), S.poll(bad)
    S.close()
    assert rb["state"] == "failed"
    assert rg["state"] == "done" and rg["steps"] == 300
    assert np.array_equal(rg["up_mean"], r_alone["up_mean"])


def test_serving_groups_requests_by_subcycle_counts():
    """Requests with other (n_int, n_DEM) run in the batch of their own class
    beside the others (no box shares a batch with other subcycle counts); all
    of them complete with the steps they asked for."""
    dps = _dps()
    kw = dict(max_steps=200, window=100, rel_tol=1e-9)
    wl, _ = _request(dps, 10, 0.1, 6)
    cs = [dps.closure(g=wl["g"], h_c=1.0, **{**KW, "n_int": ni, "n_dem": nd}) for ni, nd in ((2, 3), (3, 2), (2, 3))]
    S = dps.Server("f32", max_boxes=4, hbm_reserve_bytes=1 << 30, chunk_steps=50)
    ids = [S.submit(wl["n"], wl["periodic"], wl["tau"], wl["x"], wl["d"], wl["rho_p"], c, **kw) for c in cs]
    S.wait_idle(600)
    res = [S.poll(i) for i in ids]
    st = S.stats()
    S.close()
    assert all(r["state"] == "done" and r["steps"] == 200 for r in res), res
    assert st["failed"] == 0
    assert st["peak_boxes"] == 3  # the classes ran side by side
    # the same request in the same class gives the same result
    assert np.array_equal(res[0]["up_mean"], res[2]["up_mean"])
    assert not np.array_equal(res[0]["up_mean"], res[1]["up_mean"])


def test_read_back_of_a_box_added_after_stepping():
    """Particle read-back reads the current particle set of a stepped box from
    the device table, and the host copy of a box added since: both give the
    state in insertion order, and the late box then steps as it would alone."""
    dps = _dps()
    wls = _boxes()
    steps = 4
    B = dps.Batch("f64")
    a = B.add_box(wls[0]["n"], wls[0]["periodic"], wls[0]["tau"], len(wls[0]["x"]))
    B.add_particles(a, wls[0]["x"], wls[0]["d"], wls[0]["rho_p"])
    B.set_closure(a, _closure(dps, wls[0]))
    B.step(steps)
    ra = B.read_particles(a)
    ref_a, _ = _alone(dps, wls[0], "f64", steps)
    assert np.array_equal(ra["x"], ref_a["x"]) and np.array_equal(ra["w"], ref_a["w"])
    wl = wls[2]
    b = B.add_box(wl["n"], wl["periodic"], wl["tau"], len(wl["x"]))
    B.add_particles(b, wl["x"], wl["d"], wl["rho_p"])
    B.set_closure(b, _closure(dps, wl))
    rb = B.read_particles(b)  # not yet in the device table
    assert np.array_equal(rb["x"], np.asarray(wl["x"], dtype=np.float64))
    assert not rb["u"].any() and not rb["w"].any()
    assert np.array_equal(B.read_particles(a)["x"], ra["x"])  # the stepped box is unchanged
    B.step(steps)
    ref_b, _ = _alone(dps, wl, "f64", steps)
    got = B.read_particles(b)
    for k in ("x", "u", "w", "F"):
        assert np.array_equal(got[k], ref_b[k]), k
    B.close()
