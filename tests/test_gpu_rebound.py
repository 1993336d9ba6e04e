"""A heavy sphere thrown at the bottom wall of a closed box through a viscous
fluid (the setting of Sec. 5): the GPU trajectory through approach,
lubrication, contact and rebound follows the FP64 oracle, and lubrication
lowers the rebound (Table 3, B4 against B0)."""
import numpy as np
import pytest

import oracle as O

from test_gpu_parity import _dps, close

pytestmark = pytest.mark.gpu

SETUP = dict(n=(12, 12, 24), per=(0, 0, 0), tau=0.505, d=0.5, rho_p=32.0, x=(6.0, 6.0, 2.0), u=(0, 0, -0.03))
CL = dict(g=(0, 0, -1e-4), e_n=0.97, mu_c=0.1, T_c=0.5, h_min=1e-5, C_am=0.5, n_int=10, n_dem=50, lub_limiter=1,
          lub_cap=0.25, eps_min=0.05)


def _gpu_run(steps, **kw):
    dps = _dps()
    s = SETUP
    dom = dps.Domain(s["n"], s["per"], s["tau"], "f64", max_particles=1)
    dom.add_particles([s["x"]], [s["d"]], [s["rho_p"]], u=[s["u"]])
    dom.set_closure(fb_mode=0, skin=0.5, **{**CL, **kw})
    z, u = [], []
    for _ in range(steps):
        dom.step(1)
        p = dom.read_particles()
        z.append(p["x"][0, 2])
        u.append(p["u"][0, 2])
    dom.close()
    return np.array(z), np.array(u)


def _oracle_run(steps, **kw):
    s = SETUP
    P = O.make_params(s["n"], s["per"], s["tau"], **{**CL, **kw})
    dom = O.Domain(P, x=[s["x"]], u=[s["u"]], d=[s["d"]], rho_p=[s["rho_p"]])
    z, u = [], []
    for _ in range(steps):
        dom.step(1)
        z.append(dom.x[0, 2])
        u.append(dom.u[0, 2])
    return np.array(z), np.array(u)


def test_wall_rebound_follows_the_oracle():
    zg, ug = _gpu_run(100, h_c=0.5)
    zo, uo = _oracle_run(100, h_c=0.5)
    assert ug.max() > 0.005  # it did rebound within the window
    close(zg, zo, rtol=1e-11, what="z")
    close(ug, uo, rtol=1e-10, what="u_z")


def test_lubrication_lowers_the_rebound():
    e = {}
    for name, kw in (("wet", dict(h_c=0.5)), ("dry", dict(lubrication=0))):
        _, u = _gpu_run(100, **kw)
        k = int(np.argmax(u > 0))
        e[name] = u[k:].max() / -u[k - 1]
    assert 0.85 < e["dry"] < 1.0
    assert 0.05 < e["wet"] < e["dry"] - 0.1
