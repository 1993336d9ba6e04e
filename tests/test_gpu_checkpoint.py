"""Checkpoint / resume through the C ABI: N steps, save, destroy, a new domain
(or batch box), load, N steps must give exactly (bit for bit) what 2N
uninterrupted steps give -- every PDF, field and particle -- in every
precision form, at both AA parities of the save, and a checkpoint of another
geometry or form must be refused."""
import numpy as np
import pytest

from paper_1711_00336_gb300 import workloads

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "ubar", "u_f", "eps_f", "f_ext", "p", "f_pf", "gradP", "DuDt")


def _dps():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00336_gb300 import build, dps
    build.build()
    return dps


def _setup(dps, prec, n, per, count, seed, closure):
    pr = workloads.random_particles(n, per, count, seed, d_range=(0.8, 1.0), speed=0.005)
    pr["x"] = workloads.rsa(n, per, count, 1.0, seed, margin=0.05)  # no overlaps at the start
    dom = dps.Domain(n, per, 0.7, prec, max_particles=count + 5)
    dom.add_particles(pr["x"], pr["d"], pr["rho_p"], u=pr["u"], w=pr["w"])
    dom.set_closure(**closure)
    return dom


def _snapshot(dom):
    out = {"pdf": dom.read_pdfs()}
    out.update(dom.read_fields(FIELDS))
    out.update({"p_" + k: v for k, v in dom.read_particles().items()})
    st = dom.stats()
    out["step"] = np.array([st["step"]])
    out["counters"] = np.array([st["n_eps_clamp"], st["n_lub_limited"]])
    return out


def _assert_identical(a, b):
    for k in a:
        assert a[k].shape == b[k].shape, k
        assert np.array_equal(a[k], b[k]), f"{k}: max diff {np.abs(a[k] - b[k]).max():.3e}"


CLOSURE = dict(g=(0.0, 0.0, -2e-3), fb_mode=0, e_n=0.9, mu_c=0.25, T_c=10.0 / 6, h_c=0.6, h_min=1e-5, C_am=0.5,
               n_int=2, n_dem=3, lub_limiter=1, lub_cap=0.25, eps_min=0.05, skin=0.5)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("first", [3, 4])  # odd: saved at the odd AA parity
def test_resume_equals_uninterrupted_run(prec, first):
    dps = _dps()
    n, per, count = (14, 12, 16), (1, 1, 0), 120
    closures = dict(CLOSURE, lift=1, eilers=1, smagorinsky=1)
    ref = _setup(dps, prec, n, per, count, 31, closures)
    ref.step(first + 3)
    want = _snapshot(ref)
    ref.close()

    a = _setup(dps, prec, n, per, count, 31, closures)
    a.step(first)
    buf = a.save_state()
    a.close()
    b = dps.Domain(n, per, 0.7, prec, max_particles=count + 5)  # a fresh domain, no particles, no closure
    b.load_state(buf)
    assert b.np == count
    b.step(3)
    _assert_identical(want, _snapshot(b))
    b.close()


def test_resume_of_a_periodic_suspension_with_contacts():
    """dense triply periodic box (contacts and lubrication every substep)"""
    dps = _dps()
    wl = workloads.settling_box(L=16, eps=0.3, d=1.2, seed=9, tau=0.6)
    cl = dict(g=wl["g"], fb_mode=1, e_n=0.88, mu_c=0.25, T_c=0.5, h_c=1.2, h_min=1e-5, C_am=0.5, n_int=3,
              n_dem=4, lub_limiter=1, lub_cap=0.25, eps_min=0.05, skin=0.5)

    def make():
        dom = dps.Domain(wl["n"], wl["periodic"], wl["tau"], "f64", max_particles=len(wl["x"]))
        dom.add_particles(wl["x"], wl["d"], wl["rho_p"])
        dom.set_closure(**cl)
        return dom

    ref = make()
    ref.step(10)
    want = _snapshot(ref)
    ref.close()
    a = make()
    a.step(5)
    buf = a.save_state()
    a.close()
    b = dps.Domain(wl["n"], wl["periodic"], wl["tau"], "f64", max_particles=len(wl["x"]))
    b.load_state(buf)
    b.step(5)
    _assert_identical(want, _snapshot(b))
    b.close()


def test_batch_box_resumes_at_the_other_parity():
    """a box saved after an odd number of steps, restored into a batch that
    stands at the even parity (its PDFs moved to the other layout)"""
    dps = _dps()
    n, per, count = (12, 10, 14), (1, 0, 1), 60
    pr = workloads.random_particles(n, per, count, 5, d_range=(0.8, 1.0), speed=0.005)
    pr["x"] = workloads.rsa(n, per, count, 1.0, 5, margin=0.05)

    def batch_with_box():
        B = dps.Batch("f64")
        b = B.add_box(n, per, 0.7, count)
        B.add_particles(b, pr["x"], pr["d"], pr["rho_p"], u=pr["u"], w=pr["w"])
        B.set_closure(b, **CLOSURE)
        return B, b

    R, rb = batch_with_box()
    R.step(5)
    want = R.read_particles(rb)
    want_f = R.read_fields(rb, FIELDS)
    R.close()
    A, ab = batch_with_box()
    A.step(3)
    buf = A.save_box(ab)
    A.close()
    # the new batch holds another box that has stepped twice: parity even
    C = dps.Batch("f64")
    other = C.add_box((8, 8, 8), (1, 1, 1), 0.7, 0)
    C.set_closure(other, **CLOSURE)
    C.step(2)
    cb = C.add_box(n, per, 0.7, count)
    C.load_box(cb, buf)
    C.step(2)
    got = C.read_particles(cb)
    got_f = C.read_fields(cb, FIELDS)
    C.close()
    for k in want:
        assert np.array_equal(want[k], got[k]), k
    for k in want_f:
        assert np.array_equal(want_f[k], got_f[k]), k


def test_load_refuses_another_geometry_or_form():
    dps = _dps()
    a = _setup(dps, "f64", (10, 10, 10), (1, 1, 1), 20, 3, CLOSURE)
    a.step(1)
    buf = a.save_state()
    a.close()
    for n, per, prec, cap in [((10, 10, 11), (1, 1, 1), "f64", 25), ((10, 10, 10), (1, 1, 0), "f64", 25),
                              ((10, 10, 10), (1, 1, 1), "f32", 25), ((10, 10, 10), (1, 1, 1), "f64", 10)]:
        b = dps.Domain(n, per, 0.7, prec, max_particles=cap)
        with pytest.raises(dps.DPSError) as e:
            b.load_state(buf)
        assert e.value.code == -1  # DPS_ERR_ARG
        b.close()
    b = dps.Domain((10, 10, 10), (1, 1, 1), 0.7, "f64", max_particles=25)
    with pytest.raises(dps.DPSError):
        b.load_state(buf[:len(buf) // 2])  # truncated
    with pytest.raises(dps.DPSError):
        b.load_state(np.zeros(4096, np.uint8))  # not a checkpoint
    b.close()
