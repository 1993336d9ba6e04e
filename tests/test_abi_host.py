"""Host-side checks of the C ABI (no GPU): the library builds, loads, exports
every function that include/dps.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dps_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_1711_00336_gb300 import build, dps
    build.build()
    return dps.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "dps_step" in names and "dps_create_domain" in names
    for nm in names:
        assert hasattr(L, nm), nm


def test_version_and_lattice(L):
    from paper_1711_00336_gb300 import dps
    assert b"sm_103a" in L.dps_version()
    c, w = dps.lattice()
    assert abs(w.sum() - 1) < 1e-15
    assert (c.sum(0) == 0).all()
    # each velocity appears once, with its opposite
    s = {tuple(v) for v in c}
    assert len(s) == 19 and all(tuple(-v) in s for v in c)


def test_create_rejects_bad_descriptions_without_a_gpu(L):
    from paper_1711_00336_gb300 import dps
    h = ctypes.c_void_p()
    d = dps.DomainDesc()
    d.n[:] = [4, 4, 4]
    d.periodic[:] = [1, 1, 1]
    d.tau, d.rho_f, d.precision = 0.5, 1.0, 0  # tau must exceed 1/2
    assert L.dps_create_domain(ctypes.byref(d), ctypes.byref(h)) == -1
    assert b"tau" in L.dps_last_error(None)
    d.tau, d.precision = 0.8, 7
    assert L.dps_create_domain(ctypes.byref(d), ctypes.byref(h)) == -1
    d.precision, d.n[0] = 0, 0
    assert L.dps_create_domain(ctypes.byref(d), ctypes.byref(h)) == -1
    assert not h.value


def test_allocation_failure_is_reported_as_oom(L):
    """An allocator hook that refuses every request: create fails with
    DPS_ERR_OOM before any kernel runs (the host fault injection path)."""
    from paper_1711_00336_gb300 import dps
    calls = []

    def fail_alloc(nbytes, ctx):
        calls.append(nbytes)
        return None

    def nop_free(ptr, ctx):
        calls.append(-1)

    fa, ff = dps._ALLOC_FN(fail_alloc), dps._FREE_FN(nop_free)
    d = dps.DomainDesc()
    d.n[:] = [8, 8, 8]
    d.periodic[:] = [1, 1, 1]
    d.tau, d.rho_f, d.precision, d.max_particles = 0.8, 1.0, 0, 10
    d.alloc, d.free = fa, ff
    h = ctypes.c_void_p()
    assert L.dps_create_domain(ctypes.byref(d), ctypes.byref(h)) == -2
    assert b"allocation" in L.dps_last_error(None)
    assert calls and not h.value


def test_closure_defaults_follow_the_paper(L):
    from paper_1711_00336_gb300 import dps
    c = dps.closure()
    # Sec. 4.1: mu_c 0.25, e_n 0.88, T_c = dt/2, n_int 10, n_DEM 50; Table 1 C_am 0.5
    assert (c.mu_c, c.e_n, c.T_c, c.n_int, c.n_dem, c.C_am) == (0.25, 0.88, 0.5, 10, 50, 0.5)
    assert c.h_min == 1e-5  # Sec. 3.1.3
