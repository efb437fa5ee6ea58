"""Python binding of libdgswe (include/dgswe.h): argument marshalling only.

Every computation runs in the CUDA library.  Importing this module does not
load the library; the first Solver (or an explicit ``lib()``) does, and it
raises if ``libdgswe.so`` has not been built (``__graft_entry__.build()`` or
``python paper_2303_11767_gb300/build.py``).  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgswe.so")

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ENONFINITE, DG_ENONPHYSICAL, DG_ETIMEOUT, DG_EUNSUPPORTED = range(8)
STATUS_NAMES = {0: "DG_OK", 1: "DG_EINVAL", 2: "DG_ENOMEM", 3: "DG_ECUDA", 4: "DG_ENONFINITE",
                5: "DG_ENONPHYSICAL", 6: "DG_ETIMEOUT", 7: "DG_EUNSUPPORTED"}
PREC = {"fp64": 0, "fp32": 1, "fp32_tc_bf16": 2, "fp32_tc_fp16": 3, "fp32_tc_bf16x3": 4, "fp32_tc_fp16x3": 5}
OPT_PRECISION, OPT_RK_ORDER, OPT_CHECK_FINITE, OPT_ALPHA_MODE, OPT_STREAM, OPT_STEPS_PER_GRAPH = 1, 2, 3, 4, 5, 6
OPT_TILE_ROWS, OPT_BLOCKS_PER_SM, OPT_WELL_BALANCED = 7, 8, 9

EARTH_RADIUS = 6.37122e6
GRAVITY = 9.80616
OMEGA = 7.292e-5

# every entry point of include/dgswe.h: name -> (restype, argtypes)
_dp = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p
SIGNATURES = {
    "dg_set_device": (ctypes.c_int, [ctypes.c_int]),
    "dg_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    "dg_create_plane_advection": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "dg_create_plane_swe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    "dg_destroy": (ctypes.c_int, [_H]),
    "dg_set_option": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_longlong]),
    "dg_state_len": (ctypes.c_size_t, [_H]),
    "dg_set_state": (ctypes.c_int, [_H, _dp, ctypes.c_size_t]),
    "dg_get_state": (ctypes.c_int, [_H, _dp, ctypes.c_size_t]),
    "dg_set_state_device": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
    "dg_get_state_device": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
    "dg_rhs": (ctypes.c_int, [_H, _dp, _dp, ctypes.c_size_t]),
    "dg_step": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double]),
    "dg_total_mass": (ctypes.c_int, [_H, _dp]),
    "dg_total_mass_device": (ctypes.c_int, [_H, ctypes.c_void_p]),
    "dg_max_dt": (ctypes.c_int, [_H, ctypes.c_double, _dp]),
    "dg_projection_nodes": (ctypes.c_int, [_H, _dp, ctypes.c_size_t, _dp, ctypes.c_size_t]),
    "dg_project_nodal": (ctypes.c_int, [_H, _dp, ctypes.c_size_t, _dp, ctypes.c_size_t]),
    "dg_get_time": (ctypes.c_int, [_H, _dp]),
    "dg_set_time": (ctypes.c_int, [_H, ctypes.c_double]),
    "dg_stage_launches": (ctypes.c_longlong, [_H]),
    "dg_max_dt_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "dg_last_error": (ctypes.c_char_p, [_H]),
    "dg_measure_fp64_peak": (ctypes.c_int, [ctypes.c_int, _dp]),
    "dg_tc_check_contraction": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "dg_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                     ctypes.POINTER(ctypes.c_void_p)]),
    "dg_mlp_destroy": (ctypes.c_int, [_H]),
    "dg_mlp_num_params": (ctypes.c_size_t, [_H]),
    "dg_mlp_get_params": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
    "dg_mlp_set_params": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
    "dg_mlp_set_normalization": (ctypes.c_int, [_H] + [ctypes.POINTER(ctypes.c_float)] * 4),
    "dg_mlp_set_row_normalization": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                                    ctypes.POINTER(ctypes.c_float)]),
    "dg_mlp_forward": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "dg_mlp_gradients": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_float), ctypes.c_size_t, _dp]),
    "dg_mlp_train_step": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _dp]),
    "dg_attach_mlp": (ctypes.c_int, [_H, _H]),
    "dg_restrict_from": (ctypes.c_int, [_H, _H]),
    "dg_ensemble_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    "dg_ensemble_destroy": (ctypes.c_int, [_H]),
    "dg_ensemble_set_option": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_longlong]),
    "dg_ensemble_state_len": (ctypes.c_size_t, [_H, ctypes.c_int]),
    "dg_ensemble_total_dof": (ctypes.c_size_t, [_H]),
    "dg_ensemble_set_state": (ctypes.c_int, [_H, ctypes.c_int, _dp, ctypes.c_size_t]),
    "dg_ensemble_get_state": (ctypes.c_int, [_H, ctypes.c_int, _dp, ctypes.c_size_t]),
    "dg_ensemble_set_dt": (ctypes.c_int, [_H, _dp, ctypes.c_int]),
    "dg_ensemble_step": (ctypes.c_int, [_H, ctypes.c_int]),
    "dg_ensemble_total_mass": (ctypes.c_int, [_H, ctypes.c_int, _dp]),
    "dg_ensemble_max_dt": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double, _dp]),
    "dg_ensemble_autotune": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), _dp]),
    "dg_ensemble_stage_launches": (ctypes.c_longlong, [_H]),
    "dg_create_band": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "dg_band_halo_len": (ctypes.c_size_t, [_H]),
    "dg_band_set_reference_depth": (ctypes.c_int, [_H, ctypes.c_double]),
    "dg_band_pack": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p]),
    "dg_band_unpack": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p]),
    "dg_band_stage": (ctypes.c_int, [_H, ctypes.c_double]),
    "dg_band_mass_pair": (ctypes.c_int, [_H, _dp, _dp]),
    "dg_band_cfl_terms": (ctypes.c_int, [_H, _dp, _dp]),
}

_lib = None


class DGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib(path: str = LIB_PATH):
    """Load libdgswe.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libdgswe.so not built at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _check(status, h=None):
    if status != DG_OK:
        msg = lib().dg_last_error(h)
        raise DGError(status, msg.decode() if msg else "")


def set_device(device: int):
    _check(lib().dg_set_device(int(device)))


def measure_fp64_peak(reps: int = 5) -> float:
    """Measured FP64 FMA rate of the current device, GFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(lib().dg_measure_fp64_peak(int(reps), ctypes.byref(v)))
    return v.value


def tc_contraction_shape(degree: int, op: int):
    """(n1, k1): padded output columns and input modes of the tensor-core
    eval/trace contraction of this degree (op 0 BF16, 1 FP16)."""
    n1, k1 = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().dg_tc_check_contraction(int(degree), int(op), None, None, ctypes.byref(n1), ctypes.byref(k1)))
    return n1.value, k1.value


def tc_check_contraction(degree: int, op: int, a_dev, out_dev):
    """D = A * B1 on the tensor cores for device FP32 tensors a [128, k1] and
    out [128, n1] (torch tensors or raw device pointers)."""
    n1, k1 = ctypes.c_int(0), ctypes.c_int(0)
    pa = a_dev.data_ptr() if hasattr(a_dev, "data_ptr") else int(a_dev)
    po = out_dev.data_ptr() if hasattr(out_dev, "data_ptr") else int(out_dev)
    _check(lib().dg_tc_check_contraction(int(degree), int(op), ctypes.c_void_p(pa), ctypes.c_void_p(po),
                                         ctypes.byref(n1), ctypes.byref(k1)))
    return n1.value, k1.value


class Solver:
    """One mesh, one resident state (see include/dgswe.h for the semantics)."""

    def __init__(self, nlon, nlat, degree, radius=EARTH_RADIUS, g=GRAVITY, omega=OMEGA, precision="fp64",
                 rk_order=3, check_finite=True):
        L = lib()
        h = ctypes.c_void_p()
        _check(L.dg_create(int(nlon), int(nlat), int(degree), float(radius), float(g), float(omega),
                           ctypes.byref(h)))
        self._h = h
        self.nlon, self.nlat, self.degree = int(nlon), int(nlat), int(degree)
        self.n = self.degree + 1
        self.nphi = self.n * self.n
        self.nm = self.degree + 9
        self.radius, self.g, self.omega = float(radius), float(g), float(omega)
        self.nfields = 3
        self.set_option(OPT_PRECISION, PREC[precision] if isinstance(precision, str) else int(precision))
        self.set_option(OPT_RK_ORDER, rk_order)
        self.set_option(OPT_CHECK_FINITE, int(bool(check_finite)))

    @classmethod
    def band(cls, nlon, nlat, j_begin, j_end, degree, radius=EARTH_RADIUS, g=GRAVITY, omega=OMEGA,
             precision="fp64", rk_order=3, check_finite=True):
        """Rows [j_begin, j_end) of the nlon x nlat mesh (dg_create_band);
        state shape (j_end - j_begin, nlon, 3, (p+1)^2)."""
        self = cls.__new__(cls)
        h = ctypes.c_void_p()
        _check(lib().dg_create_band(int(nlon), int(nlat), int(j_begin), int(j_end), int(degree), float(radius),
                                    float(g), float(omega), ctypes.byref(h)))
        self._h = h
        self.nlon, self.nlat, self.degree = int(nlon), int(j_end) - int(j_begin), int(degree)
        self.j_begin, self.j_end, self.nlat_global = int(j_begin), int(j_end), int(nlat)
        self.n = self.degree + 1
        self.nphi = self.n * self.n
        self.nm = self.degree + 9
        self.radius, self.g, self.omega = float(radius), float(g), float(omega)
        self.nfields = 3
        self.set_option(OPT_PRECISION, PREC[precision] if isinstance(precision, str) else int(precision))
        self.set_option(OPT_RK_ORDER, rk_order)
        self.set_option(OPT_CHECK_FINITE, int(bool(check_finite)))
        return self

    @property
    def halo_len(self):
        """Values of one halo message (dg_band_halo_len)."""
        return int(lib().dg_band_halo_len(self._h))

    def set_reference_depth(self, href):
        _check(lib().dg_band_set_reference_depth(self._h, float(href)), self._h)

    def pack(self, side, t):
        """Boundary row (side 0 south, 1 north) of the next stage's input into
        the contiguous device tensor t (halo_len values of the working type)."""
        assert t.is_contiguous() and t.numel() == self.halo_len
        _check(lib().dg_band_pack(self._h, int(side), ctypes.c_void_p(t.data_ptr())), self._h)

    def unpack(self, side, t):
        """A neighbour's packed row into the south (0) / north (1) ghost row."""
        assert t.is_contiguous() and t.numel() == self.halo_len
        _check(lib().dg_band_unpack(self._h, int(side), ctypes.c_void_p(t.data_ptr())), self._h)

    def stage(self, dt):
        """The next RK stage of the current step (dg_band_stage)."""
        _check(lib().dg_band_stage(self._h, float(dt)), self._h)

    def cfl_terms(self):
        """(H, c) of the CFL step over this handle's rows (dg_band_cfl_terms)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().dg_band_cfl_terms(self._h, ctypes.byref(a), ctypes.byref(b)), self._h)
        return a.value, b.value

    def mass_pair(self):
        """(sum, err): the band's mass is radius^2 (sum + err)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().dg_band_mass_pair(self._h, ctypes.byref(a), ctypes.byref(b)), self._h)
        return a.value, b.value

    @classmethod
    def plane_advection(cls, nx, ny, degree, bx=1.0, by=1.0, alpha_speed=False, rk_order=4, check_finite=True):
        """The paper's planar validation problem: du/dt + div(beta u) = 0 on the
        periodic unit square, FP64; state shape (ny, nx, 1, (p+1)^2)."""
        self = cls.__new__(cls)
        h = ctypes.c_void_p()
        _check(lib().dg_create_plane_advection(int(nx), int(ny), int(degree), float(bx), float(by),
                                               int(bool(alpha_speed)), ctypes.byref(h)))
        self._h = h
        self.nlon, self.nlat, self.degree = int(nx), int(ny), int(degree)
        self.n = self.degree + 1
        self.nphi = self.n * self.n
        self.nm = self.degree + 9
        self.radius, self.g, self.omega = 1.0, 0.0, 0.0
        self.nfields = 1
        self.set_option(OPT_RK_ORDER, rk_order)
        self.set_option(OPT_CHECK_FINITE, int(bool(check_finite)))
        return self

    @classmethod
    def plane_swe(cls, nx, ny, degree, L=1.0e7, g=GRAVITY, f=1.0e-4, rk_order=4, check_finite=True):
        """Shallow water on the f-plane, [0, L]^2 periodic, FP64; state shape
        (ny, nx, 3, (p+1)^2)."""
        self = cls.__new__(cls)
        h = ctypes.c_void_p()
        _check(lib().dg_create_plane_swe(int(nx), int(ny), int(degree), float(L), float(g), float(f),
                                         ctypes.byref(h)))
        self._h = h
        self.nlon, self.nlat, self.degree = int(nx), int(ny), int(degree)
        self.n = self.degree + 1
        self.nphi = self.n * self.n
        self.nm = self.degree + 9
        self.radius, self.g, self.omega = 1.0, float(g), 0.0
        self.nfields = 3
        self.set_option(OPT_RK_ORDER, rk_order)
        self.set_option(OPT_CHECK_FINITE, int(bool(check_finite)))
        return self

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().dg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- options and sizes
    def set_option(self, key, value):
        _check(lib().dg_set_option(self._h, int(key), int(value)), self._h)

    @property
    def state_len(self):
        return int(lib().dg_state_len(self._h))

    @property
    def shape(self):
        return (self.nlat, self.nlon, self.nfields, self.nphi)

    def _host(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        if u.size != self.state_len:
            raise ValueError(f"state has {u.size} values, expected {self.state_len}")
        return u

    # -- state
    def set_state(self, u):
        u = self._host(u)
        _check(lib().dg_set_state(self._h, _ptr(u), u.size), self._h)

    def get_state(self):
        out = np.empty(self.state_len)
        _check(lib().dg_get_state(self._h, _ptr(out), out.size), self._h)
        return out.reshape(self.shape)

    def set_state_device(self, t):
        """t: contiguous float64 CUDA tensor with state_len values."""
        assert t.dtype.itemsize == 8 and t.is_contiguous() and t.numel() == self.state_len
        _check(lib().dg_set_state_device(self._h, ctypes.c_void_p(t.data_ptr()), t.numel()), self._h)

    def get_state_device(self, t):
        assert t.dtype.itemsize == 8 and t.is_contiguous() and t.numel() == self.state_len
        _check(lib().dg_get_state_device(self._h, ctypes.c_void_p(t.data_ptr()), t.numel()), self._h)

    def get_time(self):
        t = ctypes.c_double()
        _check(lib().dg_get_time(self._h, ctypes.byref(t)), self._h)
        return t.value

    def set_time(self, t):
        _check(lib().dg_set_time(self._h, float(t)), self._h)

    # -- the method
    def rhs(self, u):
        u = self._host(u)
        out = np.empty_like(u)
        _check(lib().dg_rhs(self._h, _ptr(u), _ptr(out), u.size), self._h)
        return out.reshape(self.shape)

    def step(self, n, dt):
        _check(lib().dg_step(self._h, int(n), float(dt)), self._h)

    def total_mass(self):
        m = ctypes.c_double()
        _check(lib().dg_total_mass(self._h, ctypes.byref(m)), self._h)
        return m.value

    def total_mass_device(self, t):
        """Enqueue the mass reduction; writes one float64 into CUDA tensor t."""
        _check(lib().dg_total_mass_device(self._h, ctypes.c_void_p(t.data_ptr())), self._h)

    def max_dt(self, cfl):
        dt = ctypes.c_double()
        _check(lib().dg_max_dt(self._h, float(cfl), ctypes.byref(dt)), self._h)
        return dt.value

    def stage_launches(self):
        return int(lib().dg_stage_launches(self._h))

    def attach_mlp(self, mlp):
        """Add the network's output as a learned modal source (None detaches)."""
        _check(lib().dg_attach_mlp(self._h, mlp._h if mlp is not None else None), self._h)
        self._mlp = mlp

    def restrict_from(self, fine):
        """This (coarse) solver's state := projection of `fine`'s state."""
        _check(lib().dg_restrict_from(self._h, fine._h), self._h)

    # -- projection of point values
    def projection_nodes(self):
        lam = np.empty(self.nlon * self.nm)
        th = np.empty(self.nlat * self.nm)
        _check(lib().dg_projection_nodes(self._h, _ptr(lam), lam.size, _ptr(th), th.size), self._h)
        return lam, th

    def project_nodal(self, vals):
        v = np.ascontiguousarray(vals, dtype=np.float64).reshape(-1)
        out = np.empty(self.state_len)
        _check(lib().dg_project_nodal(self._h, _ptr(v), v.size, _ptr(out), out.size), self._h)
        return out.reshape(self.shape)

    def project_grid(self, fn_grid):
        """Project fields given on the tensor grid of projection nodes:
        fn_grid(lam1, th1) -> arrays shaped [len(th1), len(lam1)], one per
        field (on the planar problems lam1, th1 are the x and y nodes)."""
        lam, th = self.projection_nodes()
        nm = self.nm
        vals = [np.asarray(v, dtype=np.float64).reshape(self.nlat, nm, self.nlon, nm).transpose(0, 2, 1, 3)
                for v in fn_grid(lam, th)][:self.nfields]
        return self.project_nodal(np.ascontiguousarray(np.stack(vals, axis=2)))


class Ensemble:
    """A batch of independent meshes advanced together (FP32, SSP-RK3); see
    include/dgswe.h."""

    def __init__(self, nlon, nlat, degree, radius=EARTH_RADIUS, g=GRAVITY, omega=OMEGA):
        L = lib()
        nm = len(nlon)
        self.nlon, self.nlat, self.degree = list(map(int, nlon)), list(map(int, nlat)), list(map(int, degree))
        arr = ctypes.c_int * nm
        h = ctypes.c_void_p()
        _check(L.dg_ensemble_create(nm, arr(*self.nlon), arr(*self.nlat), arr(*self.degree), float(radius),
                                    float(g), float(omega), ctypes.byref(h)))
        self._h = h
        self.members = nm
        self.radius = float(radius)

    def close(self):
        if getattr(self, "_h", None):
            lib().dg_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, key, value):
        _check(lib().dg_ensemble_set_option(self._h, int(key), int(value)), self._h)

    def state_len(self, m):
        return int(lib().dg_ensemble_state_len(self._h, int(m)))

    def shape(self, m):
        n = self.degree[m] + 1
        return (self.nlat[m], self.nlon[m], 3, n * n)

    @property
    def total_dof(self):
        return int(lib().dg_ensemble_total_dof(self._h))

    def set_state(self, m, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        _check(lib().dg_ensemble_set_state(self._h, int(m), _ptr(u), u.size), self._h)

    def get_state(self, m):
        out = np.empty(self.state_len(m))
        _check(lib().dg_ensemble_get_state(self._h, int(m), _ptr(out), out.size), self._h)
        return out.reshape(self.shape(m))

    def set_dt(self, dt):
        d = np.ascontiguousarray(dt, dtype=np.float64)
        _check(lib().dg_ensemble_set_dt(self._h, _ptr(d), d.size), self._h)

    def step(self, n):
        _check(lib().dg_ensemble_step(self._h, int(n)), self._h)

    def total_mass(self, m):
        x = ctypes.c_double()
        _check(lib().dg_ensemble_total_mass(self._h, int(m), ctypes.byref(x)), self._h)
        return x.value

    def max_dt(self, m, cfl):
        x = ctypes.c_double()
        _check(lib().dg_ensemble_max_dt(self._h, int(m), float(cfl), ctypes.byref(x)), self._h)
        return x.value

    def autotune(self, trials=3):
        w, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().dg_ensemble_autotune(self._h, int(trials), ctypes.byref(w), ctypes.byref(b), ctypes.byref(ms)),
               self._h)
        return w.value, b.value, ms.value

    def stage_launches(self):
        return int(lib().dg_ensemble_stage_launches(self._h))


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class MLP:
    """The per-element network of the learned correction (include/dgswe.h).
    Device batches are float32 CUDA tensors (anything with data_ptr())."""

    def __init__(self, n_in=60, n_hidden=128, n_out=12, seed=0):
        h = ctypes.c_void_p()
        _check(lib().dg_mlp_create(int(n_in), int(n_hidden), int(n_out), int(seed), ctypes.byref(h)))
        self._h = h
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)

    def close(self):
        if getattr(self, "_h", None):
            lib().dg_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(lib().dg_mlp_num_params(self._h))

    def get_params(self):
        out = np.empty(self.num_params, dtype=np.float32)
        _check(lib().dg_mlp_get_params(self._h, _fptr(out), out.size))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().dg_mlp_set_params(self._h, _fptr(p), p.size))

    def set_normalization(self, in_mean, in_std, out_mean, out_std):
        a = [np.ascontiguousarray(x, dtype=np.float32) for x in (in_mean, in_std, out_mean, out_std)]
        _check(lib().dg_mlp_set_normalization(self._h, *[_fptr(x) for x in a]))

    def set_row_normalization(self, out_mean_rows, out_std_rows):
        """Per-latitude-row output statistics [nlat, n_out] for the learned
        source; None removes them."""
        if out_mean_rows is None:
            _check(lib().dg_mlp_set_row_normalization(self._h, 0, None, None))
            return
        m = np.ascontiguousarray(out_mean_rows, dtype=np.float32)
        sd = np.ascontiguousarray(out_std_rows, dtype=np.float32)
        _check(lib().dg_mlp_set_row_normalization(self._h, int(m.shape[0]), _fptr(m), _fptr(sd)))

    def forward(self, x, y):
        _check(lib().dg_mlp_forward(self._h, ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                    ctypes.c_void_p(y.data_ptr())))

    def gradients(self, x, t):
        g = np.empty(self.num_params, dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().dg_mlp_gradients(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                      int(x.shape[0]), _fptr(g), g.size, ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, x, t, lr):
        loss = ctypes.c_double()
        _check(lib().dg_mlp_train_step(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                       int(x.shape[0]), float(lr), ctypes.byref(loss)))
        return loss.value
