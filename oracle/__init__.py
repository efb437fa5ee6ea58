"""ctypes wrapper of the FP64 CPU oracle (``dg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the CPU-baseline leg of the benchmark, never by the CUDA library or its
Python binding.  The oracle is a plain, slow FP64 implementation of the modal
DG discretisation of the shallow water equations on the sphere (arxiv
2303.11767, Sec. 2) that shares no code with the CUDA path.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
RHS_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, _dp, _dp)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_create_sphere.restype = ctypes.c_void_p
        L.oracle_create_sphere.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_create_plane_advection.restype = ctypes.c_void_p
        L.oracle_create_plane_swe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double]
        L.oracle_create_plane_swe.restype = ctypes.c_void_p
        L.oracle_create_plane_advection.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_set_alpha_mode.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_set_well_balanced.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.oracle_set_well_balanced.restype = ctypes.c_int
        L.oracle_set_alpha_mode.restype = ctypes.c_int
        L.oracle_state_len.restype = ctypes.c_size_t
        L.oracle_state_len.argtypes = [ctypes.c_void_p]
        L.oracle_nm.restype = ctypes.c_int
        L.oracle_nm.argtypes = [ctypes.c_void_p]
        L.oracle_rhs.restype = ctypes.c_int
        L.oracle_rhs.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_rhs_magnitude.restype = ctypes.c_int
        L.oracle_rhs_magnitude.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_rhs_element.restype = ctypes.c_int
        L.oracle_rhs_element.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_int, _dp]
        L.oracle_rhs_magnitude_element.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_int, _dp]
        L.oracle_rhs_magnitude_element.restype = ctypes.c_int
        L.oracle_step.restype = ctypes.c_int
        L.oracle_step.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int]
        L.oracle_rk_step.restype = ctypes.c_int
        L.oracle_rk_step.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_size_t, _dp, RHS_CB,
                                     ctypes.c_void_p]
        L.oracle_total_mass.restype = ctypes.c_double
        L.oracle_total_mass.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_max_dt.restype = ctypes.c_double
        L.oracle_max_dt.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double]
        L.oracle_projection_points.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_project.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_eval_projection_points.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_l2_error.restype = ctypes.c_double
        L.oracle_l2_error.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_int]
        L.oracle_mass_matrix.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        L.oracle_gauss_legendre.restype = ctypes.c_int
        L.oracle_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
        L.oracle_legendre.restype = ctypes.c_double
        L.oracle_legendre.argtypes = [ctypes.c_int, ctypes.c_double]
        L.oracle_legendre_deriv.restype = ctypes.c_double
        L.oracle_legendre_deriv.argtypes = [ctypes.c_int, ctypes.c_double]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().oracle_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def legendre(k: int, x: float) -> float:
    return lib().oracle_legendre(k, float(x))


def legendre_deriv(k: int, x: float) -> float:
    return lib().oracle_legendre_deriv(k, float(x))


def rk_step(order: int, dt: float, u: np.ndarray, f) -> np.ndarray:
    """One explicit RK step of the Butcher tableau of the given order applied to
    du/dt = f(u); f maps a numpy vector to a numpy vector."""
    u = np.ascontiguousarray(u, dtype=np.float64).copy()
    n = u.size

    def cb(_user, y, k):
        yy = np.ctypeslib.as_array(y, shape=(n,))
        kk = np.ctypeslib.as_array(k, shape=(n,))
        kk[:] = f(yy.copy())
        return 0

    st = lib().oracle_rk_step(order, dt, n, _ptr(u), RHS_CB(cb), None)
    if st:
        raise OracleError(f"rk_step status {st}")
    return u


class Oracle:
    """One mesh of the oracle.  State layout [row j][column i][field f][mode m],
    mode m = b*(p+1) + a (a: degree in lambda / x, b: degree in theta / y)."""

    def __init__(self, handle, nx, ny, p, nf):
        if not handle:
            raise OracleError("oracle_create failed")
        self._h = ctypes.c_void_p(handle)
        self.nx, self.ny, self.p, self.nf = nx, ny, p, nf
        self.n = p + 1
        self.nphi = self.n * self.n
        self.nm = lib().oracle_nm(self._h)

    @classmethod
    def sphere(cls, nlon, nlat, p, R=6.37122e6, g=9.80616, omega=7.292e-5):
        return cls(lib().oracle_create_sphere(nlon, nlat, p, R, g, omega), nlon, nlat, p, 3)

    @classmethod
    def plane_advection(cls, nx, ny, p, bx=1.0, by=1.0, alpha_speed=False):
        """alpha_speed: Rusanov alpha = |beta| (True) or |beta . n| (False)."""
        return cls(lib().oracle_create_plane_advection(nx, ny, p, bx, by, int(alpha_speed)), nx, ny, p, 1)

    @classmethod
    def plane_swe(cls, nx, ny, p, L=1.0e7, g=9.80616, f=1.0e-4):
        """Shallow water on the f-plane, [0, L]^2 periodic (h, hu, hv)."""
        h = lib().oracle_create_plane_swe(nx, ny, p, L, g, f)
        if not h:
            raise ValueError("invalid planar shallow-water parameters")
        return cls(h, nx, ny, p, 3)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oracle_destroy(self._h)
            self._h = None

    @property
    def state_len(self):
        return self.nx * self.ny * self.nf * self.nphi

    @property
    def shape(self):
        return (self.ny, self.nx, self.nf, self.nphi)

    def set_threads(self, n: int):
        lib().oracle_set_threads(self._h, int(n))

    def set_alpha_mode(self, mode: int):
        """0: local Rusanov alpha (default); 1: the global speeds of the stage input."""
        if lib().oracle_set_alpha_mode(self._h, int(mode)) != 0:
            raise ValueError(f"alpha mode {mode} not available for this oracle")

    def set_well_balanced(self, href: float):
        """href > 0: remove the tendency of the fluid at rest at depth href
        from every tendency (that state becomes exactly steady); 0: off."""
        if lib().oracle_set_well_balanced(self._h, float(href)) != 0:
            raise ValueError("well-balanced option not available for this oracle")

    def _in(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        if u.size != self.state_len:
            raise OracleError("bad state length")
        return u

    def rhs(self, u):
        u = self._in(u)
        out = np.empty_like(u)
        st = lib().oracle_rhs(self._h, _ptr(u), _ptr(out))
        if st:
            raise OracleError(f"rhs status {st}")
        return out.reshape(self.shape)

    def rhs_magnitude(self, u):
        """|M^-1| sum |terms| of every tendency value: the scale of the rounding
        error of any floating-point evaluation of the tendency."""
        u = self._in(u)
        out = np.empty_like(u)
        st = lib().oracle_rhs_magnitude(self._h, _ptr(u), _ptr(out))
        if st:
            raise OracleError(f"rhs_magnitude status {st}")
        return out.reshape(self.shape)

    def rhs_element(self, u, j, i):
        u = self._in(u)
        out = np.empty(self.nf * self.nphi)
        st = lib().oracle_rhs_element(self._h, _ptr(u), int(j), int(i), _ptr(out))
        if st:
            raise OracleError(f"rhs_element status {st}")
        return out.reshape(self.nf, self.nphi)

    def rhs_magnitude_element(self, u, j, i):
        """The magnitude bound of one element's tendency."""
        u = self._in(u)
        out = np.empty(self.nf * self.nphi)
        st = lib().oracle_rhs_magnitude_element(self._h, _ptr(u), int(j), int(i), _ptr(out))
        if st:
            raise OracleError(f"rhs_magnitude_element status {st}")
        return out.reshape(self.nf, self.nphi)

    def step(self, u, nsteps, dt, order=3):
        u = self._in(u).copy()
        st = lib().oracle_step(self._h, _ptr(u), int(nsteps), float(dt), int(order))
        if st:
            raise OracleError(f"step status {st}")
        return u.reshape(self.shape)

    def total_mass(self, u):
        return lib().oracle_total_mass(self._h, _ptr(self._in(u)))

    def max_dt(self, u, cfl):
        return lib().oracle_max_dt(self._h, _ptr(self._in(u)), float(cfl))

    def mass_matrix(self, j):
        m = np.empty((self.nphi, self.nphi))
        lib().oracle_mass_matrix(self._h, int(j), _ptr(m))
        return m

    def projection_points(self):
        """(x, y) of the projection points, each shaped [j][i][qy][qx]."""
        npts = self.nx * self.ny * self.nm * self.nm
        x = np.empty(npts)
        y = np.empty(npts)
        lib().oracle_projection_points(self._h, _ptr(x), _ptr(y))
        shp = (self.ny, self.nx, self.nm, self.nm)
        return x.reshape(shp), y.reshape(shp)

    def project(self, vals):
        """vals shaped [j][i][f][qy][qx] at the projection points -> modal state."""
        v = np.ascontiguousarray(vals, dtype=np.float64).reshape(-1)
        assert v.size == self.nx * self.ny * self.nf * self.nm * self.nm
        out = np.empty(self.state_len)
        lib().oracle_project(self._h, _ptr(v), _ptr(out))
        return out.reshape(self.shape)

    def project_fn(self, fn):
        """Project fn(x, y) -> array [nf, ...] (or a list of nf arrays)."""
        x, y = self.projection_points()
        vals = np.stack([np.asarray(v, dtype=np.float64) for v in fn(x, y)], axis=2)
        return self.project(vals)

    def project_tensor(self, fn_grid):
        """Project a field given on the tensor grid of projection points:
        fn_grid(x1, y1) -> nf arrays shaped [len(y1), len(x1)], where x1 runs
        over (column i, point qx) and y1 over (row j, point qy)."""
        x, y = self.projection_points()
        x1 = x[0, :, 0, :].reshape(-1)
        y1 = y[:, 0, :, 0].reshape(-1)
        nm = self.nm
        vals = [np.asarray(v, dtype=np.float64).reshape(self.ny, nm, self.nx, nm).transpose(0, 2, 1, 3)
                for v in fn_grid(x1, y1)]
        return self.project(np.ascontiguousarray(np.stack(vals, axis=2)))

    def eval_projection_points(self, u):
        out = np.empty(self.nx * self.ny * self.nf * self.nm * self.nm)
        lib().oracle_eval_projection_points(self._h, _ptr(self._in(u)), _ptr(out))
        return out.reshape(self.ny, self.nx, self.nf, self.nm, self.nm)

    def l2_error(self, u, exact_vals, field):
        ex = np.ascontiguousarray(exact_vals, dtype=np.float64).reshape(-1)
        return lib().oracle_l2_error(self._h, _ptr(self._in(u)), _ptr(ex), int(field))
