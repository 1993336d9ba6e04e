"""ctypes binding of the C ABI in ``include/dps.h`` (argument marshalling only).

Every step of the coupled method runs in the CUDA library ``libdps.so``; this
module converts numpy arrays and keyword arguments into the C structs and
pointers the ABI takes.  PyTorch provides the CUDA stream and, through the
allocator hooks, the device memory of a domain.  There is no CPU fallback: if
the library is missing or CUDA is unavailable the calls raise.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdps.so")

DPS_OK = 0
ERRORS = {-1: "DPS_ERR_ARG", -2: "DPS_ERR_OOM", -3: "DPS_ERR_STATE", -4: "DPS_ERR_UNSTABLE",
          -5: "DPS_ERR_TIMEOUT", -6: "DPS_ERR_CUDA"}
PRECISION = {"f64": 0, "f32": 1, "f16s": 2}
FIELDS = [("rho", 0x001, 1), ("ubar", 0x002, 3), ("u_f", 0x004, 3), ("eps_f", 0x008, 1),
          ("f_ext", 0x010, 3), ("p", 0x020, 1), ("f_pf", 0x040, 3), ("gradP", 0x080, 3),
          ("DuDt", 0x100, 3)]

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class DomainDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("periodic", ctypes.c_int * 3), ("tau", ctypes.c_double),
                ("rho_f", ctypes.c_double), ("precision", ctypes.c_int), ("max_particles", ctypes.c_int64),
                ("stream", ctypes.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN),
                ("alloc_ctx", ctypes.c_void_p)]


class Closure(ctypes.Structure):
    _fields_ = [("drag", ctypes.c_int), ("pressure", ctypes.c_int), ("added_mass", ctypes.c_int),
                ("lubrication", ctypes.c_int), ("contact", ctypes.c_int), ("g", ctypes.c_double * 3),
                ("fb_mode", ctypes.c_int), ("fb", ctypes.c_double * 3), ("e_n", ctypes.c_double),
                ("mu_c", ctypes.c_double), ("T_c", ctypes.c_double), ("h_c", ctypes.c_double),
                ("h_min", ctypes.c_double), ("C_am", ctypes.c_double), ("n_int", ctypes.c_int),
                ("n_dem", ctypes.c_int), ("lub_limiter", ctypes.c_int), ("lub_cap", ctypes.c_double),
                ("eps_min", ctypes.c_double), ("skin", ctypes.c_double), ("lift", ctypes.c_int),
                ("eilers", ctypes.c_int), ("smagorinsky", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("fluid_j", ctypes.c_double * 3),
                ("fluid_ubar", ctypes.c_double * 3), ("uf_mean", ctypes.c_double * 3),
                ("particle_momentum", ctypes.c_double * 3), ("up_mean", ctypes.c_double * 3),
                ("u_pS", ctypes.c_double * 3), ("eps_min_seen", ctypes.c_double),
                ("step", ctypes.c_int64), ("n_particles", ctypes.c_int64),
                ("n_eps_clamp", ctypes.c_int64), ("n_lub_limited", ctypes.c_int64),
                ("status", ctypes.c_int)]


class DPSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)


def lib():
    """Load libdps.so (build it first with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        L.dps_version.restype = ctypes.c_char_p
        L.dps_last_error.restype = ctypes.c_char_p
        L.dps_last_error.argtypes = [ctypes.c_void_p]
        L.dps_create_domain.argtypes = [ctypes.POINTER(DomainDesc), ctypes.POINTER(ctypes.c_void_p)]
        for name in ("dps_destroy", "dps_prepare", "dps_check", "dps_sync"):
            getattr(L, name).argtypes = [ctypes.c_void_p]
        for name in ("dps_step", "dps_step_async", "dps_collide_stream"):
            getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.dps_add_particles.argtypes = [ctypes.c_void_p, ctypes.c_int64, _DP, _DP, _DP, _DP, _DP]
        L.dps_write_particles.argtypes = [ctypes.c_void_p, ctypes.c_int64, _DP, _DP, _DP]
        L.dps_set_closure.argtypes = [ctypes.c_void_p, ctypes.POINTER(Closure)]
        L.dps_closure_defaults.argtypes = [ctypes.POINTER(Closure)]
        L.dps_closure_defaults.restype = None
        L.dps_read_fields.argtypes = [ctypes.c_void_p, ctypes.c_uint32, _DP, ctypes.c_int64]
        L.dps_write_fields.argtypes = [ctypes.c_void_p, ctypes.c_uint32, _DP, ctypes.c_int64]
        L.dps_read_pdfs.argtypes = [ctypes.c_void_p, _DP, ctypes.c_int64]
        L.dps_write_pdfs.argtypes = [ctypes.c_void_p, _DP, ctypes.c_int64]
        L.dps_read_particles.argtypes = [ctypes.c_void_p, _DP, _DP, _DP, _DP, ctypes.c_int64]
        L.dps_stats_get.argtypes = [ctypes.c_void_p, ctypes.POINTER(Stats)]
        L.dps_read_cell_list.argtypes = [ctypes.c_void_p, _I32P, _I32P, ctypes.c_int64, ctypes.c_int64]
        L.dps_bin_edge.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
        L.dps_lattice.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.dps_lattice.restype = None
        L.dps_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.dps_collect_timing.argtypes = [ctypes.c_void_p]
        L.dps_get_timing.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.dps_launches_per_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        L.dps_read_neighbor_list.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), _I32P, ctypes.c_int64]
        L.dps_state_size.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
        L.dps_save_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
        L.dps_load_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
        L.dps_op_cell_sort.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _vec(a, n):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, np.float64).reshape(n, 3))


def lattice():
    """(c[19,3], w[19]) in the PDF plane order of the library."""
    c = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    lib().dps_lattice(ctypes.byref(c), ctypes.byref(w))
    return np.array(list(c)).reshape(19, 3), np.array(list(w))


def closure(**kw):
    """A Closure with the library defaults, overridden by keyword arguments."""
    c = Closure()
    lib().dps_closure_defaults(ctypes.byref(c))
    for k, v in kw.items():
        if k in ("g", "fb"):
            getattr(c, k)[:] = [float(x) for x in v]
        elif k in dict(Closure._fields_):
            t = dict(Closure._fields_)[k]
            setattr(c, k, int(v) if t is ctypes.c_int else float(v))
        else:
            raise KeyError(k)
    return c


class Domain:
    """One box of the coupled method on the GPU (owner of all its device state)."""

    def __init__(self, n, periodic, tau, precision="f64", max_particles=0, rho_f=1.0, stream=None,
                 allocator="torch"):
        import torch
        L = lib()
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the dps library has no CPU path")
        self.n = tuple(int(v) for v in n)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        d = DomainDesc()
        d.n[:] = list(self.n)
        d.periodic[:] = [int(bool(v)) for v in periodic]
        d.tau, d.rho_f = float(tau), float(rho_f)
        d.precision = PRECISION[precision]
        d.max_particles = int(max_particles)
        d.stream = self.stream.cuda_stream
        self._keep = []
        if allocator == "torch":
            dev = torch.cuda.current_device()
            strm = self.stream

            def _alloc(nbytes, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)
                except Exception:
                    return None

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
            self._keep += [fa, ff]
            d.alloc, d.free = fa, ff
        self.desc = d
        h = ctypes.c_void_p()
        rc = L.dps_create_domain(ctypes.byref(d), ctypes.byref(h))
        if rc != DPS_OK:
            raise DPSError(rc, L.dps_last_error(None).decode())
        self.h = h
        self.np = 0

    def _ck(self, rc):
        if rc != DPS_OK:
            raise DPSError(rc, lib().dps_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().dps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- particles ----
    def add_particles(self, x, d, rho_p, u=None, w=None):
        x = _vec(x, -1)
        m = len(x)
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(d, np.float64), (m,)))
        rho_p = np.ascontiguousarray(np.broadcast_to(np.asarray(rho_p, np.float64), (m,)))
        self._ck(lib().dps_add_particles(self.h, m, _p(x), _p(_vec(u, m)), _p(_vec(w, m)), _p(d), _p(rho_p)))
        self.np += m

    def write_particles(self, x=None, u=None, w=None):
        m = self.np
        self._ck(lib().dps_write_particles(self.h, m, _p(_vec(x, m)), _p(_vec(u, m)), _p(_vec(w, m))))

    def read_particles(self):
        m = self.np
        out = {k: np.zeros((max(m, 1), 3)) for k in ("x", "u", "w", "F")}
        self._ck(lib().dps_read_particles(self.h, _p(out["x"]), _p(out["u"]), _p(out["w"]), _p(out["F"]),
                                          max(m, 1)))
        return {k: v[:m] for k, v in out.items()}

    # ---- closure / stepping ----
    def set_closure(self, c=None, **kw):
        c = c if c is not None else closure(**kw)
        self._ck(lib().dps_set_closure(self.h, ctypes.byref(c)))

    def prepare(self):
        self._ck(lib().dps_prepare(self.h))

    def step(self, n=1):
        self._ck(lib().dps_step(self.h, int(n)))

    def step_async(self, n=1):
        self._ck(lib().dps_step_async(self.h, int(n)))

    def check(self):
        self._ck(lib().dps_check(self.h))

    def collide_stream(self, n=1):
        self._ck(lib().dps_collide_stream(self.h, int(n)))

    def sync(self):
        self._ck(lib().dps_sync(self.h))

    # ---- tracing ----
    PHASES = ("moments+fields", "force_am", "reaction_am", "force_drag", "reaction_drag", "dem_substep",
              "cell_sort", "eps_gather", "collide_stream")

    def set_timing(self, on=True):
        self._ck(lib().dps_set_timing(self.h, int(bool(on))))

    def collect_timing(self):
        self._ck(lib().dps_collect_timing(self.h))

    def get_timing(self, reset=True):
        ms = (ctypes.c_double * 9)()
        nl = (ctypes.c_int64 * 9)()
        self._ck(lib().dps_get_timing(self.h, ctypes.byref(ms), ctypes.byref(nl), int(bool(reset))))
        return {k: {"ms": ms[i], "launches": nl[i]} for i, k in enumerate(self.PHASES)}

    def launches_per_step(self):
        n = ctypes.c_int64()
        self._ck(lib().dps_launches_per_step(self.h, ctypes.byref(n)))
        return n.value

    @property
    def search_radius(self):
        r = ctypes.c_int()
        self._ck(lib().dps_bin_edge(self.h, ctypes.byref(r)))
        return r.value

    # ---- fields ----
    def read_fields(self, names=("rho", "ubar", "u_f", "eps_f", "f_ext", "p")):
        mask = 0
        total = 0
        for nm, bit, k in FIELDS:
            if nm in names:
                mask |= bit
                total += k
        out = np.zeros(total * self.ncell)
        self._ck(lib().dps_read_fields(self.h, mask, _p(out), out.size))
        res, off = {}, 0
        for nm, bit, k in FIELDS:
            if mask & bit:
                a = out[off:off + k * self.ncell]
                res[nm] = a.reshape(k, self.ncell) if k == 3 else a.copy()
                off += k * self.ncell
        return res

    def write_fields(self, eps_f=None, f_pf=None):
        parts, mask = [], 0
        if eps_f is not None:
            parts.append(np.asarray(eps_f, np.float64).ravel())
            mask |= 0x008
        if f_pf is not None:
            parts.append(np.asarray(f_pf, np.float64).ravel())
            mask |= 0x040
        buf = np.ascontiguousarray(np.concatenate(parts))
        self._ck(lib().dps_write_fields(self.h, mask, _p(buf), buf.size))

    def read_pdfs(self):
        out = np.zeros(19 * self.ncell)
        self._ck(lib().dps_read_pdfs(self.h, _p(out), out.size))
        return out.reshape(19, self.ncell)

    def write_pdfs(self, f):
        f = np.ascontiguousarray(np.asarray(f, np.float64).ravel())
        self._ck(lib().dps_write_pdfs(self.h, _p(f), f.size))

    def stats(self):
        s = Stats()
        self._ck(lib().dps_stats_get(self.h, ctypes.byref(s)))
        out = {}
        for name, t in Stats._fields_:
            v = getattr(s, name)
            out[name] = np.array(list(v)) if hasattr(v, "__len__") else v
        return out

    def read_neighbor_list(self):
        """DEM neighbour list (dps_read_neighbor_list): CSR (offsets[np+1], partners)."""
        off = np.zeros(self.np + 1, np.int64)
        op = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        self._ck(lib().dps_read_neighbor_list(self.h, op, None, 0))
        part = np.zeros(max(int(off[-1]), 1), np.int32)
        self._ck(lib().dps_read_neighbor_list(self.h, op, part.ctypes.data_as(_I32P), part.size))
        return off, part[:int(off[-1])]

    def save_state(self):
        """Checkpoint of the domain (dps_save_state) as a uint8 numpy array."""
        n = ctypes.c_size_t()
        self._ck(lib().dps_state_size(self.h, ctypes.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        self._ck(lib().dps_save_state(self.h, ctypes.c_void_p(buf.ctypes.data), buf.size))
        return buf

    def load_state(self, buf):
        """Restore a checkpoint written by save_state (dps_load_state)."""
        buf = np.ascontiguousarray(np.asarray(buf, np.uint8))
        self._ck(lib().dps_load_state(self.h, ctypes.c_void_p(buf.ctypes.data), buf.size))
        st = self.stats()
        self.np = int(st["n_particles"])

    def read_cell_list(self):
        cs = np.zeros(self.ncell + 1, np.int32)
        order = np.zeros(max(self.np, 1), np.int32)
        self._ck(lib().dps_read_cell_list(self.h, cs.ctypes.data_as(_I32P), order.ctypes.data_as(_I32P),
                                          cs.size, order.size))
        return cs, order[:self.np]


def probe_fp64_peak():
    """Measured FP64 FMA throughput of the current GPU in GFLOP/s."""
    L = lib()
    L.dps_probe_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double)]
    v = ctypes.c_double()
    rc = L.dps_probe_fp64_peak(ctypes.byref(v))
    if rc != DPS_OK:
        raise DPSError(rc, "dps_probe_fp64_peak failed")
    return v.value


def check_tlog(x, device=False):
    """The lubrication term's logarithm and the library log of x (float64
    array), evaluated on the host or on the current GPU: (y, y_lib)."""
    L = lib()
    L.dps_check_tlog.argtypes = [_DP, _DP, _DP, ctypes.c_int64, ctypes.c_int]
    x = np.ascontiguousarray(np.asarray(x, np.float64).ravel())
    y, yl = np.empty_like(x), np.empty_like(x)
    rc = L.dps_check_tlog(x.ctypes.data_as(_DP), y.ctypes.data_as(_DP), yl.ctypes.data_as(_DP), len(x),
                          int(bool(device)))
    if rc != DPS_OK:
        raise DPSError(rc, "dps_check_tlog failed")
    return y, yl


def op_cell_sort(n, periodic, x_dev, ids_dev, stream=None):
    """Linked-cell sort of device positions (torch float64 [np,3]) and ids
    (torch int32 [np]); returns device (cell_start[ncell+1], order[np])."""
    import torch
    npart = int(x_dev.shape[0])
    ncell = int(n[0]) * int(n[1]) * int(n[2])
    cs = torch.empty(ncell + 1, dtype=torch.int32, device=x_dev.device)
    order = torch.empty(max(npart, 1), dtype=torch.int32, device=x_dev.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    pp = (ctypes.c_int * 3)(*[int(bool(v)) for v in periodic])
    rc = lib().dps_op_cell_sort(nn, pp, 1, npart, ctypes.c_void_p(x_dev.data_ptr()),
                                ctypes.c_void_p(ids_dev.data_ptr()), ctypes.c_void_p(cs.data_ptr()),
                                ctypes.c_void_p(order.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if rc != DPS_OK:
        raise DPSError(rc, "dps_op_cell_sort failed")
    return cs, order[:npart]


# ---------------------------------------------------------------------------
# batches of boxes
# ---------------------------------------------------------------------------
class BatchDesc(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("stream", ctypes.c_void_p), ("alloc", _ALLOC_FN),
                ("free", _FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


def _declare_batch(L):
    if getattr(L, "_batch_declared", False):
        return
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, _DP
    ip3 = ctypes.POINTER(ctypes.c_int)
    L.dps_batch_create.argtypes = [ctypes.POINTER(BatchDesc), ctypes.POINTER(vp)]
    L.dps_batch_last_error.argtypes = [vp]
    L.dps_batch_last_error.restype = ctypes.c_char_p
    L.dps_batch_destroy.argtypes = [vp]
    L.dps_batch_add_box.argtypes = [vp, ip3, ip3, ctypes.c_double, ctypes.c_double, i64, ctypes.POINTER(ctypes.c_int)]
    L.dps_batch_remove_box.argtypes = [vp, ctypes.c_int]
    L.dps_batch_add_particles.argtypes = [vp, ctypes.c_int, i64, dp, dp, dp, dp, dp]
    L.dps_batch_set_closure.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Closure)]
    L.dps_batch_step.argtypes = [vp, i64]
    L.dps_batch_step_async.argtypes = [vp, i64]
    L.dps_batch_check.argtypes = [vp]
    L.dps_batch_read_particles.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp, i64]
    L.dps_batch_read_fields.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, dp, i64]
    L.dps_batch_stats.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Stats)]
    L.dps_batch_particle_mean.argtypes = [vp, ctypes.c_int, dp]
    L.dps_batch_num_boxes.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.dps_batch_set_tuning.argtypes = [vp, ip3]
    L.dps_batch_get_tuning.argtypes = [vp, ip3]
    L.dps_batch_autotune.argtypes = [vp, ctypes.c_int, dp]
    L.dps_batch_set_timing.argtypes = [vp, ctypes.c_int]
    L.dps_batch_collect_timing.argtypes = [vp]
    L.dps_batch_get_timing.argtypes = [vp, vp, vp, ctypes.c_int]
    L.dps_batch_launches_per_step.argtypes = [vp, ctypes.POINTER(i64)]
    L.dps_batch_state_size.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.dps_batch_save_box.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t]
    L.dps_batch_load_box.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t]
    L.dps_box_bytes.argtypes = [ctypes.c_int, ip3, i64, ctypes.POINTER(ctypes.c_size_t)]
    L.dps_serve_create.argtypes = [ctypes.POINTER(ServeDesc), ctypes.POINTER(vp)]
    L.dps_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(i64)]
    L.dps_serve_poll.argtypes = [vp, i64, ctypes.POINTER(Result)]
    L.dps_serve_cancel.argtypes = [vp, i64]
    L.dps_serve_wait_idle.argtypes = [vp, ctypes.c_double]
    L.dps_serve_stats_get.argtypes = [vp, ctypes.POINTER(ServeStats)]
    L.dps_serve_destroy.argtypes = [vp]
    L._batch_declared = True


def _i3(v):
    return (ctypes.c_int * 3)(*[int(x) for x in v])


class Batch:
    """Many independent boxes advanced together: one launch per phase."""

    def __init__(self, precision="f32", stream=None):
        import torch
        L = lib()
        _declare_batch(L)
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the dps library has no CPU path")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        d = BatchDesc()
        d.precision = PRECISION[precision]
        d.stream = self.stream.cuda_stream
        h = ctypes.c_void_p()
        rc = L.dps_batch_create(ctypes.byref(d), ctypes.byref(h))
        if rc != DPS_OK:
            raise DPSError(rc, L.dps_last_error(None).decode())
        self.h = h
        self.boxes = {}

    def _ck(self, rc):
        if rc != DPS_OK:
            raise DPSError(rc, lib().dps_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().dps_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_box(self, n, periodic, tau, max_particles, rho_f=1.0):
        b = ctypes.c_int()
        self._ck(lib().dps_batch_add_box(self.h, _i3(n), _i3(periodic), float(tau), float(rho_f),
                                         int(max_particles), ctypes.byref(b)))
        self.boxes[b.value] = dict(n=tuple(n), np=0)
        return b.value

    def save_box(self, box):
        """Checkpoint of one box (dps_batch_save_box) as a uint8 numpy array."""
        n = ctypes.c_size_t()
        self._ck(lib().dps_batch_state_size(self.h, int(box), ctypes.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        self._ck(lib().dps_batch_save_box(self.h, int(box), ctypes.c_void_p(buf.ctypes.data), buf.size))
        return buf

    def load_box(self, box, buf):
        """Restore a checkpoint into an existing box of the same geometry (dps_batch_load_box)."""
        buf = np.ascontiguousarray(np.asarray(buf, np.uint8))
        self._ck(lib().dps_batch_load_box(self.h, int(box), ctypes.c_void_p(buf.ctypes.data), buf.size))
        self.boxes[box]["np"] = int(self.stats(box)["n_particles"])

    def remove_box(self, box):
        self._ck(lib().dps_batch_remove_box(self.h, int(box)))
        self.boxes.pop(box, None)

    def add_particles(self, box, x, d, rho_p, u=None, w=None):
        x = _vec(x, -1)
        m = len(x)
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(d, np.float64), (m,)))
        rho_p = np.ascontiguousarray(np.broadcast_to(np.asarray(rho_p, np.float64), (m,)))
        self._ck(lib().dps_batch_add_particles(self.h, int(box), m, _p(x), _p(_vec(u, m)), _p(_vec(w, m)), _p(d),
                                               _p(rho_p)))
        self.boxes[box]["np"] += m

    def set_closure(self, box, c=None, **kw):
        c = c if c is not None else closure(**kw)
        self._ck(lib().dps_batch_set_closure(self.h, int(box), ctypes.byref(c)))

    def step(self, n=1):
        self._ck(lib().dps_batch_step(self.h, int(n)))

    def step_async(self, n=1):
        self._ck(lib().dps_batch_step_async(self.h, int(n)))

    def check(self):
        self._ck(lib().dps_batch_check(self.h))

    def read_particles(self, box):
        m = self.boxes[box]["np"]
        out = {k: np.zeros((max(m, 1), 3)) for k in ("x", "u", "w", "F")}
        self._ck(lib().dps_batch_read_particles(self.h, int(box), _p(out["x"]), _p(out["u"]), _p(out["w"]),
                                                _p(out["F"]), max(m, 1)))
        return {k: v[:m] for k, v in out.items()}

    def read_fields(self, box, names=("ubar",)):
        n = self.boxes[box]["n"]
        nc = n[0] * n[1] * n[2]
        mask, total = 0, 0
        for nm, bit, k in FIELDS:
            if nm in names:
                mask |= bit
                total += k
        out = np.zeros(total * nc)
        self._ck(lib().dps_batch_read_fields(self.h, int(box), mask, _p(out), out.size))
        res, off = {}, 0
        for nm, bit, k in FIELDS:
            if mask & bit:
                a = out[off:off + k * nc]
                res[nm] = a.reshape(k, nc) if k == 3 else a.copy()
                off += k * nc
        return res

    def stats(self, box):
        """global sums, counters and the step count of one box (dps_batch_stats)"""
        s = Stats()
        self._ck(lib().dps_batch_stats(self.h, int(box), ctypes.byref(s)))
        out = {}
        for name, t in Stats._fields_:
            v = getattr(s, name)
            out[name] = np.array(list(v)) if hasattr(v, "__len__") else v
        return out

    def particle_mean(self, box):
        u = np.zeros(3)
        self._ck(lib().dps_batch_particle_mean(self.h, int(box), _p(u)))
        return u

    def tuning(self):
        """[cell threads/block, cells/tile, particle threads/block, particles/tile, collide variant]"""
        c = (ctypes.c_int * 5)()
        self._ck(lib().dps_batch_get_tuning(self.h, c))
        return list(c)

    def set_tuning(self, cfg):
        cfg = list(cfg) + [0] * (5 - len(cfg))
        self._ck(lib().dps_batch_set_tuning(self.h, (ctypes.c_int * 5)(*cfg)))

    def autotune(self, steps=5):
        ms = np.zeros(1)
        self._ck(lib().dps_batch_autotune(self.h, int(steps), _p(ms)))
        return float(ms[0])

    def set_timing(self, on=True):
        self._ck(lib().dps_batch_set_timing(self.h, int(bool(on))))

    def collect_timing(self):
        self._ck(lib().dps_batch_collect_timing(self.h))

    def get_timing(self, reset=True):
        ms = (ctypes.c_double * 9)()
        nl = (ctypes.c_int64 * 9)()
        self._ck(lib().dps_batch_get_timing(self.h, ctypes.byref(ms), ctypes.byref(nl), int(bool(reset))))
        return {k: {"ms": ms[i], "launches": nl[i]} for i, k in enumerate(Domain.PHASES)}

    def launches_per_step(self):
        n = ctypes.c_int64()
        self._ck(lib().dps_batch_launches_per_step(self.h, ctypes.byref(n)))
        return n.value


def box_bytes(precision, n, max_particles):
    L = lib()
    _declare_batch(L)
    b = ctypes.c_size_t()
    rc = L.dps_box_bytes(PRECISION[precision], _i3(n), int(max_particles), ctypes.byref(b))
    if rc != DPS_OK:
        raise DPSError(rc, "dps_box_bytes")
    return b.value


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
class ServeDesc(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("device", ctypes.c_int), ("max_boxes", ctypes.c_int),
                ("hbm_reserve_bytes", ctypes.c_size_t), ("chunk_steps", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("periodic", ctypes.c_int * 3), ("tau", ctypes.c_double),
                ("rho_f", ctypes.c_double), ("np", ctypes.c_int64), ("x3", _DP), ("d", _DP), ("rho_p", _DP),
                ("closure", Closure), ("max_steps", ctypes.c_int64), ("window", ctypes.c_int64),
                ("rel_tol", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("capped", ctypes.c_int), ("status", ctypes.c_int),
                ("steps", ctypes.c_int64), ("up_mean", ctypes.c_double * 3), ("u_pS", ctypes.c_double * 3),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_end", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("running", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("peak_boxes", ctypes.c_int), ("cell_updates", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("wall_s", ctypes.c_double)]


REQ_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


class Server:
    """Continuous-batching server (a native worker thread owns the batch)."""

    def __init__(self, precision="f32", max_boxes=64, hbm_reserve_bytes=8 << 30, chunk_steps=50, device=0):
        L = lib()
        _declare_batch(L)
        d = ServeDesc()
        d.precision = PRECISION[precision]
        d.device = int(device)
        d.max_boxes = int(max_boxes)
        d.hbm_reserve_bytes = int(hbm_reserve_bytes)
        d.chunk_steps = int(chunk_steps)
        h = ctypes.c_void_p()
        rc = L.dps_serve_create(ctypes.byref(d), ctypes.byref(h))
        if rc != DPS_OK:
            raise DPSError(rc, "dps_serve_create")
        self.h = h

    def submit(self, n, periodic, tau, x, d, rho_p, closure_obj, max_steps=20000, window=500, rel_tol=1e-3,
               rho_f=1.0):
        x = _vec(x, -1)
        m = len(x)
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(d, np.float64), (m,)))
        rho_p = np.ascontiguousarray(np.broadcast_to(np.asarray(rho_p, np.float64), (m,)))
        r = Request()
        r.n[:] = [int(v) for v in n]
        r.periodic[:] = [int(bool(v)) for v in periodic]
        r.tau, r.rho_f, r.np = float(tau), float(rho_f), m
        r.x3, r.d, r.rho_p = _p(x), _p(d), _p(rho_p)
        r.closure = closure_obj
        r.max_steps, r.window, r.rel_tol = int(max_steps), int(window), float(rel_tol)
        i = ctypes.c_int64()
        rc = lib().dps_serve_submit(self.h, ctypes.byref(r), ctypes.byref(i))
        if rc != DPS_OK:
            raise DPSError(rc, "dps_serve_submit")
        return i.value

    def poll(self, rid):
        r = Result()
        rc = lib().dps_serve_poll(self.h, int(rid), ctypes.byref(r))
        if rc != DPS_OK:
            raise DPSError(rc, "dps_serve_poll")
        return dict(state=REQ_STATES[r.state], capped=r.capped, status=r.status, steps=r.steps,
                    up_mean=np.array(list(r.up_mean)), u_pS=np.array(list(r.u_pS)), t_submit=r.t_submit,
                    t_start=r.t_start, t_end=r.t_end)

    def cancel(self, rid):
        lib().dps_serve_cancel(self.h, int(rid))

    def wait_idle(self, timeout=-1.0):
        rc = lib().dps_serve_wait_idle(self.h, float(timeout))
        if rc != DPS_OK:
            raise DPSError(rc, "wait_idle")

    def stats(self):
        s = ServeStats()
        lib().dps_serve_stats_get(self.h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in ServeStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().dps_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
