"""Named GPU cases for profiling (ncu) and tracing: each runs one part of the
library on a synthetic input through the public binding.

    python -m paper_1711_00336_gb300.profile_cases collide --n 128 --prec f64 --steps 3
    python -m paper_1711_00336_gb300.profile_cases step --workload wall_suspension --steps 3
    python -m paper_1711_00336_gb300.profile_cases settling --L 128 --eps 0.2 --prec f32 --steps 3
"""
import argparse
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["collide", "step", "settling"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--L", type=int, default=128)
    ap.add_argument("--eps", type=float, default=0.2)
    ap.add_argument("--d", type=float, default=1.5)
    ap.add_argument("--prec", default="f64")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--workload", default="wall_suspension")
    a = ap.parse_args(argv)
    import torch
    from . import build, dps, workloads
    build.build()
    if a.case == "collide":
        n = (a.n, a.n, a.n)
        dom = dps.Domain(n, (1, 1, 1), 0.65, a.prec)
        rng = np.random.default_rng(0)
        eps = rng.uniform(0.6, 1.0, dom.ncell)
        dom.write_fields(eps_f=eps, f_pf=1e-5 * rng.standard_normal(3 * dom.ncell))
        dom.collide_stream(a.warmup)
        torch.cuda.synchronize()
        dom.collide_stream(a.steps)
    else:
        if a.case == "step":
            wl = getattr(workloads, a.workload)()
            kw = dict(n_int=1, n_dem=10, T_c=1.0, e_n=0.9, h_c=1.0, fb_mode=0)
        else:
            wl = workloads.settling_box(L=a.L, eps=a.eps, d=a.d)
            kw = dict(n_int=2, n_dem=10, T_c=0.5, e_n=0.88, h_c=a.d, fb_mode=1)
        dom = dps.Domain(wl["n"], wl["periodic"], wl["tau"], a.prec, max_particles=len(wl["x"]))
        dom.add_particles(wl["x"], wl["d"], wl["rho_p"])
        dom.set_closure(g=wl["g"], mu_c=0.25, h_min=1e-5, C_am=0.5, skin=0.5, **kw)
        dom.step(a.warmup)
        dom.step(a.steps)
    dom.sync()
    dom.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
