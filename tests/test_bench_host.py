"""Host-side arithmetic of the benchmark line (no GPU): the algorithmic bytes
per cell of the collide-stream kernel, the whole-job MLUPS of the replicas,
and the partner count that scales the DEM flop model, each against a value
worked out by hand."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_collide_stream_bytes_per_cell():
    # 19 loads + 19 stores of the PDF type, eps_f and f_pf (4 field values);
    # the FP64 coupled step also reads rho and j (4 more)
    assert bench.algorithmic_bytes_collide("f64") == 2 * 19 * 8 + 4 * 8 == 336
    assert bench.algorithmic_bytes_collide("f64", True) == 336 + 4 * 8 == 368
    assert bench.algorithmic_bytes_collide("f32") == 2 * 19 * 4 + 4 * 4 == 168
    assert bench.algorithmic_bytes_collide("f16s") == 2 * 19 * 2 + 4 * 4 == 92


def test_job_mlups_counts_every_replica():
    assert abs(bench.job_mlups(2, 262144, 100, 1000.0) - 2 * 262144 * 100 / 1.0 / 1e6) < 1e-9
    assert bench.job_mlups(1, 1000, 10, 1.0) == 10.0


def test_interacting_pairs_by_hand():
    """unordered pairs within gap h_c (each pair once) plus sphere-wall pairs"""
    d = np.ones(5)
    x = np.array([(1.0, 1.0, 1.0),    # A: B at gap 0.5, bottom wall at gap 0.5
                  (2.5, 1.0, 1.0),    # B: A, bottom wall
                  (5.0, 5.0, 4.0),    # C: nothing within 1 (walls at 3.5)
                  (7.9, 6.0, 4.0),    # D: E across the periodic x face (gap -0.5)
                  (0.4, 6.0, 4.0)])   # E: D
    n, h_c = (8, 8, 8), 1.0
    # walls on z: pairs A-B, D-E and the bottom wall of A and B
    assert bench.interacting_pairs(x, d, n, (1, 1, 0), h_c) == 2 + 2
    # fully periodic: the two sphere pairs
    assert bench.interacting_pairs(x, d, n, (1, 1, 1), h_c) == 2
    # walls on x: D and E are 7.5 apart; A (x - d/2 = 0.5) and E (-0.1)
    # reach the x = 0 face, D the x = 8 face (-0.4)
    assert bench.interacting_pairs(x, d, n, (0, 1, 1), h_c) == 1 + 3


def test_stable_subcycles_by_hand():
    """n_int keeps the explicit drag relaxation beta/m dt/n_int at or below
    1/2: worked out for one box, and growing with the solid fraction and as
    the spheres get smaller."""
    import math
    L, d, tau, rho_p = 32, 1.0, 0.55, 2.5
    V = math.pi / 6 * d ** 3

    def box(eps, dd=d):
        n = int(round(eps * L ** 3 / (math.pi / 6 * dd ** 3)))
        return dict(n=(L, L, L), d=np.full(n, dd), x=np.zeros((n, 3)), tau=tau, rho_p=np.full(n, rho_p))

    # by hand at <eps_p> = 0.3: the solid fraction a sphere sees is V/8 + 1.3 * 0.3
    wl = box(0.3)
    e = V / 8 + 1.3 * len(wl["x"]) * V / L ** 3
    A = 5.81 * e / (1 - e) ** 3 + 0.48 * e ** (1 / 3) / (1 - e) ** 4
    rate = 3 * math.pi * d * (tau - 0.5) / 3 * (1 - e) * (1 / (1 - e) ** 3 + A) / (rho_p * V)
    assert bench._stable_subcycles(wl) == max(2, math.ceil(rate / 0.5))
    ns = [bench._stable_subcycles(box(eps)) for eps in (0.01, 0.1, 0.2, 0.3, 0.4, 0.45)]
    assert ns == sorted(ns) and ns[0] == 2 and ns[-1] > ns[0]
    # the same solid fraction in smaller spheres relaxes faster (rate ~ 1/d^2)
    assert bench._stable_subcycles(box(0.3, 0.6)) > bench._stable_subcycles(wl)
